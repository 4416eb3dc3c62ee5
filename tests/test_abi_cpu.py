"""CPU checks of the C ABI library: it loads without a GPU and exports every
entry point that include/lb.h declares; argument validation needs no device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0906_3611_gb300 import build
    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        build.build()
    if not os.path.exists(build.LIB):
        pytest.skip("liblb.so not built and no nvcc")
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lb_create", "lb_init_random", "lb_step", "lb_observables", "lb_get_state",
              "lb_set_state", "lb_destroy", "lb_strerror"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_0906_3611_gb300 import lb
    assert sorted(lb.EXPORTED) == _declared()
    for name in lb.EXPORTED:
        assert callable(getattr(lb, name))


def test_state_bytes_and_validation_without_gpu(lib):
    from paper_0906_3611_gb300 import lb
    assert lb.lb_state_bytes(64, 64, lb.LB_F32) == 18 * 64 * 64 * 4
    assert lb.lb_state_bytes(67, 45, lb.LB_F64) == 18 * 45 * 96 * 8
    assert lb.lb_state_bytes(4, 64, lb.LB_F32) == 0
    assert lb.lb_state_bytes(64, 64, 9) == 0
    h = ctypes.c_void_p()
    p = lb.make_params()
    assert lib.lb_create(4, 64, ctypes.byref(p), None, ctypes.byref(h)) == lb.LB_EINVAL
    bad = lb.make_params(tau=(0.5, 1.0))
    assert lib.lb_create(64, 64, ctypes.byref(bad), None, ctypes.byref(h)) == lb.LB_EINVAL
    bad = lb.make_params(storage=7)
    assert lib.lb_create(64, 64, ctypes.byref(bad), None, ctypes.byref(h)) == lb.LB_EINVAL
    bad = lb.make_params(boundary=3)
    assert lib.lb_create(64, 64, ctypes.byref(bad), None, ctypes.byref(h)) == lb.LB_EINVAL
    bad = lb.make_params(rho0=0.0)
    assert lib.lb_create(64, 64, ctypes.byref(bad), None, ctypes.byref(h)) == lb.LB_EINVAL
    assert lib.lb_step(None, 1) == lb.LB_EINVAL
    assert lb.lb_strerror(lb.LB_ENOMEM) == "out of memory"
    assert lb.lb_time(0) == -1


def test_invalid_arguments_of_the_newer_calls_without_gpu(lib):
    """NULL handles and out-of-range arguments are refused before any device
    work (shear, response record, bursts, overlap, batch layout and state, the
    row-kernel shape calls)."""
    from paper_0906_3611_gb300 import lb
    E = lb.LB_EINVAL
    d = ctypes.c_double()
    n = ctypes.c_int64()
    hist = (ctypes.c_int64 * 4)()
    assert lib.lb_shear_diagnostics(None, ctypes.byref(d), ctypes.byref(d)) == E
    assert lib.lb_series_start(None, 16) == E
    assert lib.lb_series_read(None, ctypes.byref(d), 1, ctypes.byref(n)) == E
    assert lib.lb_series_stop(None) == E
    assert lib.lb_series_bursts(None, ctypes.c_double(2.0), 4, hist, ctypes.byref(n)) == E
    assert lib.lb_phi_snapshot(None) == E
    assert lib.lb_phi_overlap(None, ctypes.byref(d), ctypes.byref(d)) == E
    assert lib.lb_batch_set_layout(None, 0, 1) == E
    assert lib.lb_batch_set_state(None, 0, ctypes.byref(d)) == E
    assert lib.lb_batch_series_start(None, 0, 16) == E
    assert lib.lb_batch_series_read(None, 0, ctypes.byref(d), 1, ctypes.byref(n)) == E
    assert lib.lb_batch_series_stop(None, 0) == E
    assert lib.lb_batch_series_bursts(None, 0, ctypes.c_double(2.0), 4, hist, ctypes.byref(n)) == E
    shape = ctypes.c_int(7)
    assert lib.lb_row_shape(None) == -1
    assert lib.lb_autotune(None, 8, ctypes.byref(shape)) == E and shape.value == 7
    h = ctypes.c_void_p()
    for bad in (lb.make_params(g_kolmo=1e-3, k_kolmo=0), lb.make_params(g_kolmo=float("nan"))):
        assert lib.lb_create(64, 64, ctypes.byref(bad), None, ctypes.byref(h)) == E


def test_mixture_parameters_are_validated_without_gpu(lib):
    """lb_mix_create refuses bad species counts, tau_s <= 1/2, an asymmetric
    cross-coupling matrix, 16-bit storage and non-finite values before any
    device work; NULL handles are refused by every lb_mix call."""
    from paper_0906_3611_gb300 import lb
    E = lb.LB_EINVAL
    G = [[0, 0.4, 0.2], [0.4, 0, 0.3], [0.2, 0.3, 0]]
    ok = dict(ns=3, tau=[1, 1, 1], rho0=0.7, Ga=[-9, -9, 0], Gr=[8.1, 8.1, 0], G=G)
    h = ctypes.c_void_p()

    def create(**kw):
        args = dict(ok, **kw)
        return lib.lb_mix_create(64, 64, ctypes.byref(lb.make_mix_params(**args)), None,
                                 ctypes.byref(h))

    bad_G = [[0, 0.4, 0.2], [0.41, 0, 0.3], [0.2, 0.3, 0]]
    assert create(G=bad_G) == E
    assert create(tau=[1, 0.5, 1]) == E
    assert create(storage=lb.LB_F16_DEV) == E
    assert create(rho0=float("nan")) == E
    assert create(boundary=2) == E
    p5 = lb.make_mix_params(**ok)
    p5.ns = 5
    assert lib.lb_mix_create(64, 64, ctypes.byref(p5), None, ctypes.byref(h)) == E
    p1 = lb.make_mix_params(**ok)
    p1.ns = 1
    assert lib.lb_mix_create(64, 64, ctypes.byref(p1), None, ctypes.byref(h)) == E
    assert lib.lb_mix_create(4, 64, ctypes.byref(lb.make_mix_params(**ok)), None,
                             ctypes.byref(h)) == E
    assert lib.lb_mix_step(None, 1) == E
    assert lib.lb_mix_observables(None, None, None) == E
    assert lib.lb_mix_status(None) == E
    assert lib.lb_mix_sync(None) == E
