"""FP64 CPU oracle of the two-species soft-glassy lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the correctness reference for the
CUDA path (Benzi et al., arXiv:0906.3611, Sec. II: Eq. (be), Eq. (FORCE),
Eq. (PSI), Table I).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the product package and does not import it.

The arithmetic lives in ``lb_oracle.c`` (plain C, FP64, separate
whole-lattice passes); this module compiles it with gcc and wraps it with
ctypes.  ``theory.py`` holds the paper's closed forms and root-finders used
as pins.  Every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "liblb_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
COUETTE = 1
INIT_UNIFORM_NOISE = 0
INIT_BERNOULLI = 1


def build(force: bool = False) -> str:
    """Compile ``lb_oracle.c`` into ``liblb_oracle.so`` next to it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.lbo_tables.argtypes = [ip, ip, dp, ip, ip, dp, dp]
        lib.lbo_tables.restype = None
        lib.lbo_densities.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.lbo_densities.restype = None
        lib.lbo_forces.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.lbo_forces.restype = None
        lib.lbo_step.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, ctypes.c_int]
        lib.lbo_step.restype = ctypes.c_long
        lib.lbo_observables.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
        lib.lbo_observables.restype = ctypes.c_long
        lib.lbo_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.lbo_philox4x32_10.restype = None
        lib.lbo_init.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, dp]
        lib.lbo_init.restype = None
        lib.lbo_init_densities.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_int, dp, dp]
        lib.lbo_init_densities.restype = None
        lib.lbo_shear_diagnostics.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.lbo_shear_diagnostics.restype = ctypes.c_long
        lib.lbo_phi_overlap.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
        lib.lbo_phi_overlap.restype = None
        lib.lbo_densities_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.lbo_densities_ns.restype = None
        lib.lbo_forces_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.lbo_forces_ns.restype = None
        lib.lbo_step_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, ctypes.c_int]
        lib.lbo_step_ns.restype = ctypes.c_long
        lib.lbo_observables_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.lbo_observables_ns.restype = ctypes.c_long
        lib.lbo_init_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                    dp, dp]
        lib.lbo_init_ns.restype = None
        lib.lbo_max_threads.argtypes = []
        lib.lbo_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params_vector(p: dict) -> np.ndarray:
    """Pack a parameter dict into the oracle's parameter vector.

    Keys: tau (pair), rho0, G_AB, Ga (pair), Gr (pair), boundary, U_wall,
    g_kolmo (Kolmogorov body acceleration amplitude, default 0) and k_kolmo
    (its wave number, default 1).
    """
    tau = p.get("tau", (1.0, 1.0))
    Ga = p.get("Ga", (0.0, 0.0))
    Gr = p.get("Gr", (0.0, 0.0))
    return np.array([tau[0], tau[1], p.get("rho0", 1.0), p.get("G_AB", 0.0),
                     Ga[0], Ga[1], Gr[0], Gr[1], float(p.get("boundary", PERIODIC)),
                     p.get("U_wall", 0.0), p.get("g_kolmo", 0.0), float(p.get("k_kolmo", 1))],
                    dtype=np.float64)


def tables():
    """Return (cx9, cy9, w9, cxF, cyF, pF, wF) exactly as the oracle uses them."""
    lib = _load()
    cx9 = (ctypes.c_int * 9)(); cy9 = (ctypes.c_int * 9)(); w9 = (ctypes.c_double * 9)()
    cxf = (ctypes.c_int * 25)(); cyf = (ctypes.c_int * 25)()
    pf = (ctypes.c_double * 25)(); wf = (ctypes.c_double * 25)()
    lib.lbo_tables(cx9, cy9, w9, cxf, cyf, pf, wf)
    return (np.array(cx9[:]), np.array(cy9[:]), np.array(w9[:]), np.array(cxf[:]),
            np.array(cyf[:]), np.array(pf[:]), np.array(wf[:]))


def densities(f: np.ndarray) -> np.ndarray:
    """rho[2, ny, nx] of a population array f[2, 9, ny, nx]."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, _, ny, nx = f.shape
    rho = np.empty((2, ny, nx))
    lib.lbo_densities(_dp(f), nx, ny, _dp(rho))
    return rho


def forces(rho: np.ndarray, p: dict) -> np.ndarray:
    """F[2 species, 2 comps, ny, nx] of density fields rho[2, ny, nx], Eq. (FORCE)."""
    lib = _load()
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    _, ny, nx = rho.shape
    F = np.empty((2, 2, ny, nx))
    lib.lbo_forces(_dp(rho), nx, ny, _dp(params_vector(p)), _dp(F))
    return F


def step(f: np.ndarray, p: dict, nsteps: int = 1, threads: int = 0):
    """Advance a copy of f[2, 9, ny, nx] by nsteps; returns (f_new, bad_count)."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    _, _, ny, nx = g.shape
    bad = lib.lbo_step(_dp(g), nx, ny, _dp(params_vector(p)), int(nsteps), int(threads))
    if bad < 0:
        raise MemoryError("oracle step: allocation failed")
    return g, int(bad)


def observables(f: np.ndarray, p: dict) -> dict:
    """rho[2,ny,nx], u[2,ny,nx], stress[3], mass[4] of a state (see lb_oracle.c)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, _, ny, nx = f.shape
    rho = np.empty((2, ny, nx)); u = np.empty((2, ny, nx))
    stress = np.empty(3); mass = np.empty(4)
    bad = lib.lbo_observables(_dp(f), nx, ny, _dp(params_vector(p)), _dp(rho), _dp(u),
                              _dp(stress), _dp(mass))
    if bad < 0:
        raise MemoryError("oracle observables: allocation failed")
    return {"rho": rho, "u": u, "stress": stress, "mass": mass, "bad": int(bad)}


def shear_diagnostics(f: np.ndarray, p: dict) -> dict:
    """Sec. VII diagnostics of a state: U_k (sine amplitude of the line-averaged
    x velocity at the forcing wave number; R = U_k / U0) and I_AB (Eq. (INDICATOR))."""
    lib = _load()
    _, _, ny, nx = f.shape
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(2)
    bad = lib.lbo_shear_diagnostics(_dp(f), nx, ny, _dp(params_vector(p)), _dp(out))
    return {"U_k": float(out[0]), "I_AB": float(out[1]), "bad": int(bad)}


def phi_overlap(f_w: np.ndarray, f: np.ndarray) -> tuple[float, float]:
    """The two sums of the ageing overlap, Eq. (CORRE), of one realisation:
    (sum phi(t_w) phi(t_w + dt_w), sum phi(t_w)^2), phi = rho_A - rho_B, for the
    states f_w (at t_w) and f (dt_w later), both f[2, 9, ny, nx]."""
    lib = _load()
    f_w = np.ascontiguousarray(f_w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f_w.shape == f.shape
    _, _, ny, nx = f.shape
    out = np.zeros(2)
    lib.lbo_phi_overlap(_dp(f_w), _dp(f), nx, ny, _dp(out))
    return float(out[0]), float(out[1])


def overlap_C(pairs) -> float:
    """C(t_w, dt_w) of Eq. (CORRE) over an ensemble: the ratio of the two sums,
    each averaged over the realisations (pairs of (f_w, f))."""
    sums = np.array([phi_overlap(fw, f) for fw, f in pairs])
    return float(sums[:, 0].mean() / sums[:, 1].mean())


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: four 32-bit counter words, two key words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.lbo_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def init_state(nx: int, ny: int, seed: int, kind: int, init) -> np.ndarray:
    """Seeded initial populations f = w_i rho_s (zero velocity)."""
    lib = _load()
    f = np.empty((2, 9, ny, nx))
    iv = np.zeros(6)
    iv[: len(init)] = init
    lib.lbo_init(_dp(f), nx, ny, ctypes.c_uint64(seed), int(kind), _dp(iv))
    return f


def init_densities(nx: int, ny: int, seed: int, kind: int, init) -> np.ndarray:
    lib = _load()
    rho = np.empty((2, ny, nx))
    iv = np.zeros(6)
    iv[: len(init)] = init
    lib.lbo_init_densities(nx, ny, ctypes.c_uint64(seed), int(kind), _dp(iv), _dp(rho))
    return rho


# ---- N_s species (Sec. II, Eq. (be) and Eq. (FORCE) for s = 1..N_s) ----

def params_ns(p: dict) -> np.ndarray:
    """Parameter vector of the N_s-species passes.  Keys: ns, tau (ns values),
    rho0, Ga, Gr (ns values each), G (ns x ns symmetric cross couplings; the
    diagonal is not used), boundary, U_wall, g_kolmo, k_kolmo."""
    ns = int(p["ns"])
    tau = np.asarray(p.get("tau", [1.0] * ns), dtype=np.float64)
    Ga = np.asarray(p.get("Ga", [0.0] * ns), dtype=np.float64)
    Gr = np.asarray(p.get("Gr", [0.0] * ns), dtype=np.float64)
    G = np.asarray(p.get("G", np.zeros((ns, ns))), dtype=np.float64).reshape(ns, ns)
    head = [float(ns), p.get("rho0", 1.0), float(p.get("boundary", PERIODIC)), p.get("U_wall", 0.0),
            p.get("g_kolmo", 0.0), float(p.get("k_kolmo", 1))]
    return np.concatenate([np.array(head), tau, Ga, Gr, G.ravel()])


def densities_ns(f: np.ndarray) -> np.ndarray:
    """rho[ns, ny, nx] of f[ns, 9, ny, nx]."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    ns, _, ny, nx = f.shape
    rho = np.empty((ns, ny, nx))
    lib.lbo_densities_ns(_dp(f), ns, nx, ny, _dp(rho))
    return rho


def forces_ns(rho: np.ndarray, p: dict) -> np.ndarray:
    """F[ns, 2, ny, nx] of density fields rho[ns, ny, nx], Eq. (FORCE) for N_s species."""
    lib = _load()
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ns, ny, nx = rho.shape
    assert ns == int(p["ns"])
    F = np.empty((ns, 2, ny, nx))
    lib.lbo_forces_ns(_dp(rho), nx, ny, _dp(params_ns(p)), _dp(F))
    return F


def step_ns(f: np.ndarray, p: dict, nsteps: int = 1, threads: int = 0):
    """Advance a copy of f[ns, 9, ny, nx] by nsteps; returns (f_new, bad_count)."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    ns, _, ny, nx = g.shape
    assert ns == int(p["ns"])
    bad = lib.lbo_step_ns(_dp(g), nx, ny, _dp(params_ns(p)), int(nsteps), int(threads))
    if bad < 0:
        raise MemoryError("oracle step_ns: allocation failed or ns out of range")
    return g, int(bad)


def observables_ns(f: np.ndarray, p: dict) -> dict:
    """mass[ns] (per species), momentum[2], stress[3] and the bad count of a state."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    ns, _, ny, nx = f.shape
    stress = np.empty(3)
    mass = np.empty(ns + 2)
    bad = lib.lbo_observables_ns(_dp(f), nx, ny, _dp(params_ns(p)), _dp(stress), _dp(mass))
    if bad < 0:
        raise MemoryError("oracle observables_ns: allocation failed")
    return {"mass": mass[:ns], "momentum": mass[ns:], "stress": stress, "bad": int(bad)}


def init_ns(ns: int, nx: int, ny: int, seed: int, mean, amp) -> np.ndarray:
    """Seeded state at rest: rho_s = mean[s] + amp[s] (2u - 1), one Philox block
    (counter (site, 1 + s), key seed) per site and species, f = w_i rho_s."""
    lib = _load()
    f = np.empty((ns, 9, ny, nx))
    m = np.ascontiguousarray(mean, dtype=np.float64)
    a = np.ascontiguousarray(amp, dtype=np.float64)
    lib.lbo_init_ns(_dp(f), ns, nx, ny, ctypes.c_uint64(seed), _dp(m), _dp(a))
    return f


def max_threads() -> int:
    return int(_load().lbo_max_threads())
