"""Thin ctypes binding of liblb.so (include/lb.h), names as in the C ABI.

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels.  PyTorch provides device memory (the two
population buffers, via ``lb_create_on``) and CUDA streams.  If the library
is missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblb.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ETIMEOUT, LB_EBUSY, LB_ENEGRHO = 0, -1, -2, -3, -4, -5, -6
LB_ETOOBIG = -7
LB_PERIODIC, LB_COUETTE = 0, 1
LB_F64, LB_F32, LB_BF16_DEV, LB_F16_DEV = 0, 1, 2, 3
LB_INIT_UNIFORM_NOISE, LB_INIT_BERNOULLI = 0, 1
ELEM_BYTES = {LB_F64: 8, LB_F32: 4, LB_BF16_DEV: 2, LB_F16_DEV: 2}

# every entry point declared in include/lb.h
EXPORTED = ["lb_state_bytes", "lb_create", "lb_create_on", "lb_init_random", "lb_step",
            "lb_row_shape", "lb_autotune",
            "lb_observables", "lb_shear_diagnostics", "lb_series_start", "lb_series_read",
            "lb_series_stop", "lb_series_bursts", "lb_batch_series_bursts", "lb_phi_snapshot", "lb_phi_overlap",
            "lb_get_state", "lb_set_state",
            "lb_set_state_raw",
            "lb_get_state_raw", "lb_time", "lb_status", "lb_sync", "lb_destroy", "lb_strerror",
            "lb_observables_noalloc", "lb_batch_create", "lb_batch_add", "lb_batch_remove",
            "lb_batch_set_steps", "lb_batch_run", "lb_batch_poll", "lb_batch_observables",
            "lb_batch_get_state", "lb_batch_set_state",
            "lb_batch_series_start", "lb_batch_series_read", "lb_batch_series_stop", "lb_batch_shear_diagnostics", "lb_batch_phi_snapshot",
            "lb_batch_phi_overlap", "lb_batch_autotune", "lb_batch_set_layout",
            "lb_batch_status", "lb_batch_destroy",
            "lb_mix_create", "lb_mix_init_random", "lb_mix_step", "lb_mix_observables",
            "lb_mix_get_state", "lb_mix_set_state", "lb_mix_status", "lb_mix_sync",
            "lb_mix_destroy"]
LB_MAX_SPECIES = 4


class lb_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("rho0", ctypes.c_double), ("G_AB", ctypes.c_double),
                ("Ga", ctypes.c_double * 2), ("Gr", ctypes.c_double * 2), ("boundary", ctypes.c_int),
                ("U_wall", ctypes.c_double), ("storage", ctypes.c_int),
                ("rho_ref", ctypes.c_double * 2), ("init_kind", ctypes.c_int),
                ("init", ctypes.c_double * 6), ("g_kolmo", ctypes.c_double),
                ("k_kolmo", ctypes.c_int)]


class lb_mix_params(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("tau", ctypes.c_double * 4), ("rho0", ctypes.c_double),
                ("Ga", ctypes.c_double * 4), ("Gr", ctypes.c_double * 4),
                ("G", (ctypes.c_double * 4) * 4), ("boundary", ctypes.c_int),
                ("U_wall", ctypes.c_double), ("storage", ctypes.c_int)]


class LBError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lb_strerror(code)} ({code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    hp = ctypes.POINTER(vp)
    pp = ctypes.POINTER(lb_params)
    sig = {
        "lb_state_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "lb_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, pp, vp, hp]),
        "lb_create_on": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, pp, vp, vp, vp, ctypes.c_size_t, hp]),
        "lb_init_random": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "lb_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lb_row_shape": (ctypes.c_int, [vp]),
        "lb_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "lb_observables": (ctypes.c_int, [vp, dp, dp, dp, dp]),
        "lb_shear_diagnostics": (ctypes.c_int, [vp, dp, dp]),
        "lb_series_start": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lb_series_read": (ctypes.c_int, [vp, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
        "lb_series_stop": (ctypes.c_int, [vp]),
        "lb_series_bursts": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]),
        "lb_batch_series_bursts": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.POINTER(ctypes.c_int64)]),
        "lb_phi_snapshot": (ctypes.c_int, [vp]),
        "lb_phi_overlap": (ctypes.c_int, [vp, dp, dp]),
        "lb_batch_phi_snapshot": (ctypes.c_int, [vp, ctypes.c_int]),
        "lb_batch_phi_overlap": (ctypes.c_int, [vp, ctypes.c_int, dp, dp]),
        "lb_get_state": (ctypes.c_int, [vp, dp]),
        "lb_set_state": (ctypes.c_int, [vp, dp]),
        "lb_set_state_raw": (ctypes.c_int, [vp, vp]),
        "lb_get_state_raw": (ctypes.c_int, [vp, vp]),
        "lb_time": (ctypes.c_int64, [vp]),
        "lb_status": (ctypes.c_int, [vp]),
        "lb_sync": (ctypes.c_int, [vp]),
        "lb_destroy": (None, [vp]),
        "lb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lb_observables_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp,
                                                  vp, vp]),
        "lb_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, hp]),
        "lb_batch_add": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, pp, ctypes.c_uint64,
                                        ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_remove": (ctypes.c_int, [vp, ctypes.c_int]),
        "lb_batch_set_steps": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
        "lb_batch_run": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lb_batch_poll": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "lb_batch_observables": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, dp, dp]),
        "lb_batch_get_state": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lb_batch_set_state": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "lb_batch_series_start": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
        "lb_batch_series_read": (ctypes.c_int, [vp, ctypes.c_int, dp, ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_int64)]),
        "lb_batch_series_stop": (ctypes.c_int, [vp, ctypes.c_int]),
        "lb_batch_shear_diagnostics": (ctypes.c_int, [vp, ctypes.c_int, dp, dp]),
        "lb_batch_set_layout": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "lb_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]),
        "lb_batch_status": (ctypes.c_int, [vp]),
        "lb_batch_destroy": (None, [vp]),
        "lb_mix_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(lb_mix_params),
                                         vp, hp]),
        "lb_mix_init_random": (ctypes.c_int, [vp, ctypes.c_uint64, dp, dp]),
        "lb_mix_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lb_mix_observables": (ctypes.c_int, [vp, dp, dp]),
        "lb_mix_get_state": (ctypes.c_int, [vp, dp]),
        "lb_mix_set_state": (ctypes.c_int, [vp, dp]),
        "lb_mix_status": (ctypes.c_int, [vp]),
        "lb_mix_sync": (ctypes.c_int, [vp]),
        "lb_mix_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != LB_OK:
        raise LBError(rc, what)


def make_params(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1),
                boundary=LB_PERIODIC, U_wall=0.0, storage=LB_F32, rho_ref=(1.0, 1.0),
                init_kind=LB_INIT_UNIFORM_NOISE, init=(1.0, 1.0, 0.05), g_kolmo=0.0,
                k_kolmo=1) -> lb_params:
    p = lb_params()
    p.tau[:] = list(tau)
    p.rho0 = rho0
    p.G_AB = G_AB
    p.Ga[:] = list(Ga)
    p.Gr[:] = list(Gr)
    p.boundary = boundary
    p.U_wall = U_wall
    p.storage = storage
    p.rho_ref[:] = list(rho_ref)
    p.init_kind = init_kind
    iv = list(init) + [0.0] * (6 - len(init))
    p.init[:] = iv
    p.g_kolmo = g_kolmo
    p.k_kolmo = k_kolmo
    return p


# ---- the C ABI, one Python function per entry point ----

def lb_state_bytes(nx: int, ny: int, storage: int) -> int:
    return int(_lib.lb_state_bytes(nx, ny, storage))


def lb_create(nx: int, ny: int, params: lb_params, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(_lib.lb_create(nx, ny, ctypes.byref(params), ctypes.c_void_p(stream or 0),
                          ctypes.byref(h)), "lb_create")
    return h.value


def lb_create_on(nx: int, ny: int, params: lb_params, stream: int | None, buf0: int, buf1: int,
                 bytes_each: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.lb_create_on(nx, ny, ctypes.byref(params), ctypes.c_void_p(stream or 0),
                             ctypes.c_void_p(buf0), ctypes.c_void_p(buf1), bytes_each,
                             ctypes.byref(h)), "lb_create_on")
    return h.value


def lb_init_random(h: int, seed: int) -> None:
    _check(_lib.lb_init_random(h, ctypes.c_uint64(seed)), "lb_init_random")


def lb_step(h: int, n: int) -> None:
    _check(_lib.lb_step(h, n), "lb_step")


def lb_observables(h: int, rho=None, u=None, stress=None, mass=None) -> None:
    _check(_lib.lb_observables(h, _dp(rho), _dp(u), _dp(stress), _dp(mass)), "lb_observables")


def lb_shear_diagnostics(h: int) -> tuple[float, float]:
    """(U_k, I_AB) of the current state (Sec. VII)."""
    uk = np.zeros(1)
    iab = np.zeros(1)
    _check(_lib.lb_shear_diagnostics(h, _dp(uk), _dp(iab)), "lb_shear_diagnostics")
    return float(uk[0]), float(iab[0])


def lb_series_start(h: int, capacity: int) -> None:
    _check(_lib.lb_series_start(h, capacity), "lb_series_start")


def lb_series_read(h: int, max_count: int) -> np.ndarray:
    out = np.zeros(max(max_count, 1))
    n = ctypes.c_int64(0)
    _check(_lib.lb_series_read(h, _dp(out), max_count, ctypes.byref(n)), "lb_series_read")
    return out[:n.value].copy()


def lb_series_stop(h: int) -> None:
    _check(_lib.lb_series_stop(h), "lb_series_stop")


def _bursts(fn, name, args, nbins: int) -> dict:
    hist = (ctypes.c_int64 * nbins)()
    ev = ctypes.c_int64(0)
    _check(fn(*args, nbins, hist, ctypes.byref(ev)), name)
    return {"hist": np.array(list(hist), dtype=np.int64), "events": int(ev.value)}


def lb_series_bursts(h: int, c: float, nbins: int) -> dict:
    return _bursts(_lib.lb_series_bursts, "lb_series_bursts", (h, c), nbins)


def lb_batch_series_bursts(b: int, slot: int, c: float, nbins: int) -> dict:
    return _bursts(_lib.lb_batch_series_bursts, "lb_batch_series_bursts", (b, slot, c), nbins)


def lb_phi_snapshot(h: int) -> None:
    _check(_lib.lb_phi_snapshot(h), "lb_phi_snapshot")


def lb_phi_overlap(h: int) -> tuple[float, float]:
    num = np.zeros(1)
    den = np.zeros(1)
    _check(_lib.lb_phi_overlap(h, _dp(num), _dp(den)), "lb_phi_overlap")
    return float(num[0]), float(den[0])


def lb_batch_phi_snapshot(b: int, slot: int) -> None:
    _check(_lib.lb_batch_phi_snapshot(b, slot), "lb_batch_phi_snapshot")


def lb_batch_phi_overlap(b: int, slot: int) -> tuple[float, float]:
    num = np.zeros(1)
    den = np.zeros(1)
    _check(_lib.lb_batch_phi_overlap(b, slot, _dp(num), _dp(den)), "lb_batch_phi_overlap")
    return float(num[0]), float(den[0])


def lb_get_state(h: int, f: np.ndarray) -> None:
    _check(_lib.lb_get_state(h, _dp(f)), "lb_get_state")


def lb_set_state(h: int, f: np.ndarray) -> None:
    _check(_lib.lb_set_state(h, _dp(np.ascontiguousarray(f, dtype=np.float64))), "lb_set_state")


def lb_set_state_raw(h: int, ptr: int) -> None:
    _check(_lib.lb_set_state_raw(h, ctypes.c_void_p(ptr)), "lb_set_state_raw")


def lb_get_state_raw(h: int, ptr: int) -> None:
    _check(_lib.lb_get_state_raw(h, ctypes.c_void_p(ptr)), "lb_get_state_raw")


def lb_row_shape(h: int) -> int:
    return int(_lib.lb_row_shape(h))


def lb_autotune(h: int, steps_per_candidate: int) -> int:
    shape = ctypes.c_int(-1)
    _check(_lib.lb_autotune(h, steps_per_candidate, ctypes.byref(shape)), "lb_autotune")
    return shape.value


def lb_time(h: int) -> int:
    return int(_lib.lb_time(h))


def lb_status(h: int) -> int:
    return int(_lib.lb_status(h))


def lb_sync(h: int) -> None:
    _check(_lib.lb_sync(h), "lb_sync")


def lb_destroy(h: int) -> None:
    _lib.lb_destroy(h)


def lb_observables_noalloc(f_ptr: int, nx: int, ny: int, pitch: int, params: lb_params,
                           stream: int | None, out_ptr: int) -> None:
    """Observables of a device population buffer into 8 device doubles, with no
    allocation (for callers that cannot call cudaMalloc; see include/lb.h)."""
    _check(_lib.lb_observables_noalloc(ctypes.c_void_p(f_ptr), nx, ny, pitch, ctypes.byref(params),
                                       ctypes.c_void_p(stream or 0), ctypes.c_void_p(out_ptr)),
           "lb_observables_noalloc")


# ---- batched ensembles ----

def lb_batch_create(capacity: int, storage: int, stream: int | None = None) -> int:
    b = ctypes.c_void_p()
    _check(_lib.lb_batch_create(capacity, storage, ctypes.c_void_p(stream or 0), ctypes.byref(b)),
           "lb_batch_create")
    return b.value


def lb_batch_add(b: int, nx: int, ny: int, params: lb_params, seed: int, steps: int) -> int:
    slot = ctypes.c_int(-1)
    _check(_lib.lb_batch_add(b, nx, ny, ctypes.byref(params), ctypes.c_uint64(seed), steps,
                             ctypes.byref(slot)), "lb_batch_add")
    return slot.value


def lb_batch_remove(b: int, slot: int) -> None:
    _check(_lib.lb_batch_remove(b, slot), "lb_batch_remove")


def lb_batch_set_steps(b: int, slot: int, steps: int) -> None:
    _check(_lib.lb_batch_set_steps(b, slot, steps), "lb_batch_set_steps")


def lb_batch_run(b: int, n: int) -> None:
    _check(_lib.lb_batch_run(b, n), "lb_batch_run")


def lb_batch_poll(b: int, capacity: int):
    rem = (ctypes.c_int64 * capacity)()
    done = (ctypes.c_int64 * capacity)()
    _check(_lib.lb_batch_poll(b, rem, done), "lb_batch_poll")
    return np.array(rem[:]), np.array(done[:])


def lb_batch_observables(b: int, slot: int, rho=None, u=None, stress=None, mass=None) -> None:
    _check(_lib.lb_batch_observables(b, slot, _dp(rho), _dp(u), _dp(stress), _dp(mass)),
           "lb_batch_observables")


def lb_batch_get_state(b: int, slot: int, f: np.ndarray) -> None:
    _check(_lib.lb_batch_get_state(b, slot, _dp(f)), "lb_batch_get_state")


def lb_batch_series_start(b: int, slot: int, capacity: int) -> None:
    _check(_lib.lb_batch_series_start(b, slot, capacity), "lb_batch_series_start")


def lb_batch_series_read(b: int, slot: int, max_count: int) -> np.ndarray:
    out = np.zeros(max(max_count, 1))
    n = ctypes.c_int64(0)
    _check(_lib.lb_batch_series_read(b, slot, _dp(out), max_count, ctypes.byref(n)),
           "lb_batch_series_read")
    return out[:n.value].copy()


def lb_batch_series_stop(b: int, slot: int) -> None:
    _check(_lib.lb_batch_series_stop(b, slot), "lb_batch_series_stop")


def lb_batch_set_state(b: int, slot: int, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(_lib.lb_batch_set_state(b, slot, _dp(f)), "lb_batch_set_state")


def lb_batch_shear_diagnostics(b: int, slot: int) -> tuple[float, float]:
    uk = np.zeros(1)
    iab = np.zeros(1)
    _check(_lib.lb_batch_shear_diagnostics(b, slot, _dp(uk), _dp(iab)), "lb_batch_shear_diagnostics")
    return float(uk[0]), float(iab[0])


def lb_batch_set_layout(b: int, layout: int, rows_per_item: int) -> None:
    _check(_lib.lb_batch_set_layout(b, layout, rows_per_item), "lb_batch_set_layout")


def lb_batch_autotune(b: int, steps_per_candidate: int) -> tuple[int, int]:
    layout = ctypes.c_int(0)
    rows = ctypes.c_int(0)
    _check(_lib.lb_batch_autotune(b, steps_per_candidate, ctypes.byref(layout), ctypes.byref(rows)),
           "lb_batch_autotune")
    return layout.value, rows.value


def lb_batch_status(b: int) -> int:
    return int(_lib.lb_batch_status(b))


def lb_batch_destroy(b: int) -> None:
    _lib.lb_batch_destroy(b)


def lb_strerror(code: int) -> str:
    return _lib.lb_strerror(code).decode()


class Lattice:
    """One lattice on the current CUDA device, populations in torch-owned memory.

    ``params`` is an ``lb_params`` (see ``make_params``).  ``stream`` is a
    ``torch.cuda.Stream`` (default: a new one).  Device memory for the two
    population buffers comes from PyTorch and is passed to ``lb_create_on``.
    """

    def __init__(self, nx: int, ny: int, params: lb_params, stream=None, torch_buffers: bool = True):
        import torch

        self.nx, self.ny, self.params = nx, ny, params
        self.stream = stream if stream is not None else torch.cuda.Stream()
        sptr = self.stream.cuda_stream
        self.bytes_each = lb_state_bytes(nx, ny, params.storage)
        if self.bytes_each == 0:
            raise LBError(LB_EINVAL, "lb_state_bytes")
        self._bufs = None
        if torch_buffers:
            self._bufs = [torch.empty(self.bytes_each, dtype=torch.uint8, device="cuda") for _ in range(2)]
            torch.cuda.current_stream().synchronize()
            self.h = lb_create_on(nx, ny, params, sptr, self._bufs[0].data_ptr(),
                                  self._bufs[1].data_ptr(), self.bytes_each)
        else:
            self.h = lb_create(nx, ny, params, sptr)

    def init_random(self, seed: int):
        lb_init_random(self.h, seed)
        return self

    def step(self, n: int = 1):
        lb_step(self.h, n)
        return self

    @property
    def row_shape(self) -> int:
        """CTA shape of the row kernel (0, 1), -1 for the tile kernel."""
        return lb_row_shape(self.h)

    def autotune(self, steps_per_candidate: int = 8) -> int:
        """Time the row-kernel shapes and keep the fastest (state unchanged)."""
        return lb_autotune(self.h, steps_per_candidate)

    def series_start(self, capacity: int):
        """Record U_k after every step (device ring of `capacity` entries)."""
        lb_series_start(self.h, capacity)
        return self

    def series(self, max_count: int = 1 << 20) -> np.ndarray:
        """The recorded U_k, oldest first (R = U_k / U0)."""
        return lb_series_read(self.h, max_count)

    def series_stop(self):
        lb_series_stop(self.h)
        return self

    def series_bursts(self, c: float = 3.0, nbins: int = 32) -> dict:
        """Bursts of dU/dt in the record and the log2 histogram of their spacing."""
        return lb_series_bursts(self.h, c, nbins)

    def phi_snapshot(self):
        """Store phi(t_w) = rho_A - rho_B of the current state (Eq. (CORRE))."""
        lb_phi_snapshot(self.h)
        return self

    def phi_overlap(self) -> tuple[float, float]:
        """(sum phi(t_w) phi(t), sum phi(t_w)^2) for the current state t."""
        return lb_phi_overlap(self.h)

    def shear_diagnostics(self) -> dict:
        """U_k (R = U_k / U0, Eq. (RESPONSE)) and I_AB (Eq. (INDICATOR))."""
        uk, iab = lb_shear_diagnostics(self.h)
        return {"U_k": uk, "I_AB": iab}

    def observables(self, fields: bool = False) -> dict:
        stress = np.zeros(3)
        mass = np.zeros(4)
        rho = u = None
        if fields:
            rho = np.zeros((2, self.ny, self.nx))
            u = np.zeros((2, self.ny, self.nx))
        lb_observables(self.h, rho, u, stress, mass)
        out = {"stress": stress, "mass": mass}
        if fields:
            out["rho"] = rho
            out["u"] = u
        return out

    def get_state(self) -> np.ndarray:
        f = np.empty((2, 9, self.ny, self.nx))
        lb_get_state(self.h, f)
        return f

    def set_state(self, f: np.ndarray):
        lb_set_state(self.h, f)
        return self

    @property
    def time(self) -> int:
        return lb_time(self.h)

    def status(self) -> int:
        return lb_status(self.h)

    def sync(self):
        lb_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            lb_destroy(self.h)
            self.h = None
        self._bufs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batched ensemble of independent lattices (see include/lb.h, lb_batch_*)."""

    def __init__(self, capacity: int, storage: int, stream=None):
        import torch

        self.capacity = capacity
        self.storage = storage
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.h = lb_batch_create(capacity, storage, self.stream.cuda_stream)
        self.shapes = {}

    def add(self, nx: int, ny: int, params: lb_params, seed: int, steps: int) -> int:
        slot = lb_batch_add(self.h, nx, ny, params, seed, steps)
        self.shapes[slot] = (nx, ny)
        return slot

    def remove(self, slot: int):
        lb_batch_remove(self.h, slot)
        self.shapes.pop(slot, None)

    def set_steps(self, slot: int, steps: int):
        lb_batch_set_steps(self.h, slot, steps)

    def run(self, n: int):
        lb_batch_run(self.h, n)
        return self

    def poll(self):
        return lb_batch_poll(self.h, self.capacity)

    def observables(self, slot: int, fields: bool = False) -> dict:
        nx, ny = self.shapes[slot]
        stress, mass = np.zeros(3), np.zeros(4)
        rho = u = None
        if fields:
            rho, u = np.zeros((2, ny, nx)), np.zeros((2, ny, nx))
        lb_batch_observables(self.h, slot, rho, u, stress, mass)
        out = {"stress": stress, "mass": mass}
        if fields:
            out["rho"], out["u"] = rho, u
        return out

    def get_state(self, slot: int) -> np.ndarray:
        nx, ny = self.shapes[slot]
        f = np.empty((2, 9, ny, nx))
        lb_batch_get_state(self.h, slot, f)
        return f

    def series_start(self, slot: int, capacity: int):
        """Record the replica's U_k after every step (device ring of `capacity`)."""
        lb_batch_series_start(self.h, slot, capacity)
        return self

    def series(self, slot: int, max_count: int = 1 << 20) -> np.ndarray:
        """The replica's recorded U_k, oldest first (R = U_k / U0)."""
        return lb_batch_series_read(self.h, slot, max_count)

    def series_stop(self, slot: int):
        lb_batch_series_stop(self.h, slot)
        return self

    def series_bursts(self, slot: int, c: float = 3.0, nbins: int = 32) -> dict:
        return lb_batch_series_bursts(self.h, slot, c, nbins)

    def set_state(self, slot: int, f: np.ndarray):
        """Replace the replica's state by FP64 populations [2][9][ny][nx]."""
        nx, ny = self.shapes[slot]
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (2, 9, ny, nx):
            raise ValueError(f"state of shape {f.shape}, expected {(2, 9, ny, nx)}")
        lb_batch_set_state(self.h, slot, f)
        return self

    def shear_diagnostics(self, slot: int) -> dict:
        uk, iab = lb_batch_shear_diagnostics(self.h, slot)
        return {"U_k": uk, "I_AB": iab}

    def phi_snapshot(self, slot: int):
        lb_batch_phi_snapshot(self.h, slot)

    def phi_overlap(self, slot: int) -> tuple[float, float]:
        return lb_batch_phi_overlap(self.h, slot)

    def set_layout(self, layout: int, rows_per_item: int = 1 << 30):
        """Work-list layout (0 contiguous, 1 packed, 2 waves) and longest piece."""
        lb_batch_set_layout(self.h, layout, rows_per_item)
        return self

    def autotune(self, steps_per_candidate: int = 4) -> tuple[int, int]:
        """(layout, longest piece in rows) chosen by the library's autotuner."""
        return lb_batch_autotune(self.h, steps_per_candidate)

    def status(self) -> int:
        return lb_batch_status(self.h)

    def close(self):
        if getattr(self, "h", None):
            lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- mixtures of N_s species ----

def make_mix_params(ns: int, tau, rho0: float, Ga, Gr, G, boundary: int = LB_PERIODIC,
                    U_wall: float = 0.0, storage: int = LB_F32) -> lb_mix_params:
    """lb_mix_params for ns species: tau, Ga, Gr of length ns, G an ns x ns
    symmetric matrix (its diagonal is not used)."""
    p = lb_mix_params()
    p.ns = int(ns)
    for s_ in range(ns):
        p.tau[s_] = float(tau[s_])
        p.Ga[s_] = float(Ga[s_])
        p.Gr[s_] = float(Gr[s_])
        for t in range(ns):
            p.G[s_][t] = float(np.asarray(G)[s_][t])
    p.rho0 = float(rho0)
    p.boundary = int(boundary)
    p.U_wall = float(U_wall)
    p.storage = int(storage)
    return p


def lb_mix_create(nx: int, ny: int, params: lb_mix_params, stream: int | None = None) -> int:
    m = ctypes.c_void_p()
    _check(_lib.lb_mix_create(nx, ny, ctypes.byref(params), ctypes.c_void_p(stream or 0),
                              ctypes.byref(m)), "lb_mix_create")
    return m.value


def lb_mix_init_random(m: int, seed: int, mean, amp) -> None:
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    _check(_lib.lb_mix_init_random(m, ctypes.c_uint64(seed), _dp(mean), _dp(amp)),
           "lb_mix_init_random")


def lb_mix_step(m: int, n: int) -> None:
    _check(_lib.lb_mix_step(m, n), "lb_mix_step")


def lb_mix_observables(m: int, ns: int) -> tuple[np.ndarray, np.ndarray]:
    mass = np.zeros(ns)
    mom = np.zeros(2)
    _check(_lib.lb_mix_observables(m, _dp(mass), _dp(mom)), "lb_mix_observables")
    return mass, mom


def lb_mix_get_state(m: int, f: np.ndarray) -> None:
    _check(_lib.lb_mix_get_state(m, _dp(f)), "lb_mix_get_state")


def lb_mix_set_state(m: int, f: np.ndarray) -> None:
    _check(_lib.lb_mix_set_state(m, _dp(f)), "lb_mix_set_state")


def lb_mix_status(m: int) -> int:
    return int(_lib.lb_mix_status(m))


def lb_mix_sync(m: int) -> None:
    _check(_lib.lb_mix_sync(m), "lb_mix_sync")


def lb_mix_destroy(m: int) -> None:
    _lib.lb_mix_destroy(m)


class Mixture:
    """An nx x ny lattice of ns species on the current CUDA device (library-owned
    buffers); ``stream`` is a torch.cuda.Stream (default: a new one)."""

    def __init__(self, nx: int, ny: int, params: lb_mix_params, stream=None):
        import torch

        self.nx, self.ny, self.ns, self.params = nx, ny, params.ns, params
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.h = lb_mix_create(nx, ny, params, self.stream.cuda_stream)

    def init_random(self, seed: int, mean, amp):
        lb_mix_init_random(self.h, seed, mean, amp)
        return self

    def step(self, n: int = 1):
        lb_mix_step(self.h, n)
        return self

    def observables(self) -> dict:
        mass, mom = lb_mix_observables(self.h, self.ns)
        return {"mass": mass, "momentum": mom}

    def get_state(self) -> np.ndarray:
        f = np.empty((self.ns, 9, self.ny, self.nx))
        lb_mix_get_state(self.h, f)
        return f

    def set_state(self, f: np.ndarray):
        lb_mix_set_state(self.h, np.ascontiguousarray(f, dtype=np.float64))
        return self

    def status(self) -> int:
        return lb_mix_status(self.h)

    def sync(self):
        lb_mix_sync(self.h)

    def close(self):
        if self.h:
            lb_mix_destroy(self.h)
            self.h = None
