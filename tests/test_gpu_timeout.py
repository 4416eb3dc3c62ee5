"""The device-timeout path of the row-streaming kernels, exercised without
hanging anything.

Every wait of the row kernels for a staged row is bounded (about a second by
default).  LB_TEST_WAIT_CYCLES, read when a lattice or batch is created,
shortens the compute warps' bound to a few cycles: their first wait gives up
before the first bulk copy lands, the step is abandoned, the CTA's staging
warp stops issuing copies and waits (at the full bound) for the copies it
already issued, and the status word reports LB_ETIMEOUT.  A lattice created
afterwards with the default bound steps normally and matches the oracle.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _p(lb, storage):
    return lb.make_params(**CFG, boundary=lb.LB_COUETTE, U_wall=0.02, storage=storage,
                          rho_ref=(1.0, 1.0))


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 1e-4), ("f64", 1e-12)])
def test_a_wait_that_gives_up_reports_a_timeout_and_the_next_lattice_is_exact(
        lb, monkeypatch, storage, tol):
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "f64": lb.LB_F64}[storage]
    nx, ny = 1024, 96
    f = inputs.populations(nx, ny, seed=5, base=W9, rel_amp=0.02)
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    monkeypatch.setenv("LB_TEST_WAIT_CYCLES", "0")
    lat = lb.Lattice(nx, ny, _p(lb, st))
    lat.set_state(f).step(1)
    assert lat.status() == lb.LB_ETIMEOUT
    lat.step(2)  # abandoned steps again: still no fault, the context stays usable
    assert lat.status() == lb.LB_ETIMEOUT
    lat.close()
    monkeypatch.delenv("LB_TEST_WAIT_CYCLES")
    lat = lb.Lattice(nx, ny, _p(lb, st))
    f0 = lat.set_state(f).get_state()  # (the state as the storage holds it)
    g = lat.step(1).get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, _ = oracle.step(f0, dict(CFG, boundary=1, U_wall=0.02), 1)
    assert float(np.max(np.abs(g - ref) / np.abs(ref))) <= tol


def test_a_batch_whose_wait_gives_up_reports_a_timeout(lb, monkeypatch):
    monkeypatch.setenv("LB_TEST_WAIT_CYCLES", "0")
    b = lb.Batch(4, lb.LB_F32)
    for k in range(3):
        b.add(256 + 128 * k, 64, _p(lb, lb.LB_F32), k, 10)
    b.run(3)
    assert b.status() == lb.LB_ETIMEOUT
    b.close()
    monkeypatch.delenv("LB_TEST_WAIT_CYCLES")
    b = lb.Batch(4, lb.LB_F32)
    b.add(256, 64, _p(lb, lb.LB_F32), 0, 10)
    b.run(3)
    assert b.status() == lb.LB_OK
    b.close()
