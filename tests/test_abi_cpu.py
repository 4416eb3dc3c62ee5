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
