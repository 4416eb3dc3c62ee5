"""The device-timeout path of the row-streaming kernels, exercised without
hanging anything.

Every mbarrier wait of the row kernels is bounded (about a second).
LB_TEST_STALL_STAGING, read when a lattice or batch is created, makes the
kernels' staging warps issue no bulk copy at all: the compute warps' first
wait for a staged row runs out after that second, the step is abandoned, and
the status word reports LB_ETIMEOUT; later abandoned steps end the same way
and the context stays usable.  A lattice created afterwards without the hook
steps normally and matches the oracle.
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
def test_a_stalled_staging_warp_reports_a_timeout_and_the_next_lattice_is_exact(
        lb, monkeypatch, storage, tol):
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "f64": lb.LB_F64}[storage]
    nx, ny = 1024, 96
    f = inputs.populations(nx, ny, seed=5, base=W9, rel_amp=0.02)
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    monkeypatch.setenv("LB_TEST_STALL_STAGING", "1")
    lat = lb.Lattice(nx, ny, _p(lb, st))
    lat.set_state(f).step(1)
    assert lat.status() == lb.LB_ETIMEOUT
    lat.step(2)  # abandoned steps again: still no fault, the context stays usable
    assert lat.status() == lb.LB_ETIMEOUT
    lat.close()
    monkeypatch.delenv("LB_TEST_STALL_STAGING")
    lat = lb.Lattice(nx, ny, _p(lb, st))
    f0 = lat.set_state(f).get_state()  # (the state as the storage holds it)
    g = lat.step(1).get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, _ = oracle.step(f0, dict(CFG, boundary=1, U_wall=0.02), 1)
    assert float(np.max(np.abs(g - ref) / np.abs(ref))) <= tol


def test_a_batch_with_stalled_staging_reports_a_timeout(lb, monkeypatch):
    monkeypatch.setenv("LB_TEST_STALL_STAGING", "1")
    b = lb.Batch(4, lb.LB_F32)
    for k in range(3):
        b.add(256 + 128 * k, 64, _p(lb, lb.LB_F32), k, 10)
    b.run(3)
    assert b.status() == lb.LB_ETIMEOUT
    b.close()
    monkeypatch.delenv("LB_TEST_STALL_STAGING")
    b = lb.Batch(4, lb.LB_F32)
    b.add(256, 64, _p(lb, lb.LB_F32), 0, 10)
    b.run(3)
    assert b.status() == lb.LB_OK
    b.close()
