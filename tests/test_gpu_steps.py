"""The three ways a lattice is stepped agree bit for bit.

A lattice stepped n times in one call replays captured graphs of 32 steps
and launches the rest one by one; stepped one step per call, it launches
every step alone; run as a batch replica, it goes through the batched
kernel, which splits the rows into other work items.  The per-site
arithmetic does not depend on any of this, so all three must agree bit for
bit, across graph boundaries, odd step counts and the buffer parity they
leave, in every storage and for both boundaries.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
EMUL = (0.7, 1.2, 0.1, 0.02)


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _p(lb, storage, boundary):
    return lb.make_params(**CFG, boundary=boundary, U_wall=0.03 if boundary else 0.0,
                          storage=storage, rho_ref=(0.88, 0.44),
                          init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)


@pytest.mark.parametrize("boundary", [0, 1], ids=["periodic", "couette"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f64"])
def test_one_call_equals_single_steps_and_the_batched_kernel(lb, monkeypatch, storage, boundary):
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV, "f64": lb.LB_F64}[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    nx, ny, seed, n = 384, 72, 21, 131  # 131 = 4 x 32 + 3: four graph replays, odd parity
    p = _p(lb, st, boundary)
    a = lb.Lattice(nx, ny, p).init_random(seed).step(n)
    fa = a.get_state()
    assert a.status() == lb.LB_OK
    b = lb.Lattice(nx, ny, p).init_random(seed)
    for _ in range(n):
        b.step(1)
    fb = b.get_state()
    assert b.status() == lb.LB_OK
    a.close()
    b.close()
    assert np.array_equal(fa, fb)
    bt = lb.Batch(2, st)
    slot = bt.add(nx, ny, p, seed, n)
    bt.run(n)
    fc = bt.get_state(slot)
    assert bt.status() == lb.LB_OK
    bt.close()
    assert np.array_equal(fa, fc)
