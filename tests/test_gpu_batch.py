"""Batched ensembles (lb_batch_*): many lattices of uneven sizes, couplings,
boundaries and step budgets advanced by one persistent launch per step.

Each replica's result must equal the same lattice run alone through the
single-lattice row kernel bit for bit (the per-site arithmetic does not
depend on how the rows are split into work items), and FP64 replicas match
the oracle at 1e-12.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
ASYM = dict(tau=(0.8, 1.3), rho0=0.83, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
EMUL = (0.7, 1.2, 0.1, 0.02)


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _p(lb, phys, storage, boundary, U):
    # droplet emulsion for the workload couplings; the asymmetric couplings
    # start from rho = 1 +- 0.05 (droplets of them reach rho <= 0 within 20 steps)
    if phys is CFG:
        return lb.make_params(**phys, boundary=boundary, U_wall=U, storage=storage,
                              rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)
    return lb.make_params(**phys, boundary=boundary, U_wall=U, storage=storage,
                          rho_ref=(1.0, 1.0), init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(1.0, 1.0, 0.05))


def _alone(lb, monkeypatch, nx, ny, p, seed, steps):
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    lat = lb.Lattice(nx, ny, p).init_random(seed).step(steps)
    f = lat.get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    return f


REPLICAS = [  # nx, ny, physics, boundary, U, seed, budget
    (256, 64, CFG, 0, 0.0, 11, 30),
    (384, 40, ASYM, 1, 0.03, 12, 17),
    (128, 128, CFG, 1, 0.01, 13, 30),
    (64, 24, ASYM, 0, 0.0, 14, 5),
]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f64"])
def test_batch_equals_each_replica_alone(lb, monkeypatch, storage):
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV, "f64": lb.LB_F64}[storage]
    b = lb.Batch(8, st)
    slots = [b.add(nx, ny, _p(lb, ph, st, bd, U), seed, steps)
             for nx, ny, ph, bd, U, seed, steps in REPLICAS]
    b.run(32)  # two graph replays of 16 steps; every budget runs out inside them
    rem, done = b.poll()
    assert b.status() == lb.LB_OK
    for k, (nx, ny, ph, bd, U, seed, steps) in zip(slots, REPLICAS):
        assert rem[k] == 0 and done[k] == steps
        got = b.get_state(k)
        ref = _alone(lb, monkeypatch, nx, ny, _p(lb, ph, st, bd, U), seed, steps)
        assert np.array_equal(got, ref), (nx, ny)
    b.close()


def test_batch_fp64_matches_the_oracle(lb):
    b = lb.Batch(4, lb.LB_F64)
    nx, ny = 136, 30
    p = _p(lb, ASYM, lb.LB_F64, 1, 0.04)
    k = b.add(nx, ny, p, 5, 7)
    k2 = b.add(256, 16, _p(lb, CFG, lb.LB_F64, 0, 0.0), 6, 3)
    b.run(10)
    got = b.get_state(k)
    b.close()
    f0 = oracle.init_state(nx, ny, 5, oracle.INIT_UNIFORM_NOISE, (1.0, 1.0, 0.05))
    ref, _ = oracle.step(f0, dict(ASYM, boundary=1, U_wall=0.04), 7)
    scale = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :, None, None] * ref.sum(axis=1)[:, None]
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-12


def test_slots_are_reused_after_remove(lb, monkeypatch):
    b = lb.Batch(2, lb.LB_F32)
    a = b.add(256, 32, _p(lb, CFG, lb.LB_F32, 0, 0.0), 1, 4)
    c = b.add(128, 48, _p(lb, CFG, lb.LB_F32, 1, 0.02), 2, 100)
    with pytest.raises(lb.LBError):
        b.add(128, 16, _p(lb, CFG, lb.LB_F32, 0, 0.0), 3, 4)  # full
    b.run(4)
    b.remove(a)
    d = b.add(192, 20, _p(lb, ASYM, lb.LB_F32, 1, 0.05), 4, 9)
    assert d == a
    b.run(9)
    rem, done = b.poll()
    assert done[d] == 9 and done[c] == 13 and rem[c] == 87
    got_d, got_c = b.get_state(d), b.get_state(c)
    b.close()
    assert np.array_equal(got_d, _alone(lb, monkeypatch, 192, 20, _p(lb, ASYM, lb.LB_F32, 1, 0.05), 4, 9))
    assert np.array_equal(got_c, _alone(lb, monkeypatch, 128, 48, _p(lb, CFG, lb.LB_F32, 1, 0.02), 2, 13))


def test_autotune_keeps_results_exact(lb, monkeypatch):
    b = lb.Batch(4, lb.LB_F32)
    k = b.add(512, 256, _p(lb, CFG, lb.LB_F32, 1, 0.02), 7, 1000)
    layout, rows = b.autotune(2)  # 8 candidates x (2 + 1) steps
    assert (layout, rows) in ((0, 1 << 30), (0, 512), (1, 1 << 30), (1, 512), (1, 128),
                              (2, 512), (2, 256), (2, 128))
    b.run(5)
    rem, done = b.poll()
    n = int(done[k])
    assert n == 8 * 3 + 5
    got = b.get_state(k)
    obs = b.observables(k)
    b.close()
    ref = _alone(lb, monkeypatch, 512, 256, _p(lb, CFG, lb.LB_F32, 1, 0.02), 7, n)
    assert np.array_equal(got, ref)
    assert obs["mass"][0] > 0


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_set_state_of_a_replica_mid_run(lb, monkeypatch, storage):
    """lb_batch_set_state replaces one replica's state after some steps; the
    replica then continues exactly like a lattice started from that state
    (FP64: the state reads back bit for bit), and its neighbour is untouched."""
    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    import inputs
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    nx, ny = 128, 40
    f = inputs.populations(nx, ny, seed=31, base=w9, rel_amp=0.05, species_scale=(0.9, 0.45))
    if storage == "f32":
        f = f.astype(np.float32).astype(np.float64)
    p = _p(lb, CFG, st, 1, 0.02)
    q = _p(lb, ASYM, st, 0, 0.0)
    b = lb.Batch(2, st)
    k = b.add(nx, ny, p, 1, 25)
    k2 = b.add(64, 24, q, 2, 25)
    b.run(5)
    b.set_state(k, f)
    if storage == "f64":
        assert np.array_equal(b.get_state(k), f)
    b.run(20)
    got, other = b.get_state(k), b.get_state(k2)
    assert b.status() == lb.LB_OK
    b.close()
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    lat = lb.Lattice(nx, ny, p).set_state(f).step(20)
    assert np.array_equal(lat.get_state(), got)
    lat.close()
    assert np.array_equal(_alone(lb, monkeypatch, 64, 24, q, 2, 25), other)


@pytest.mark.parametrize("layout,rows", [(0, 1 << 30), (0, 7), (1, 1 << 30), (1, 33), (2, 1 << 30),
                                         (2, 256), (2, 5)])
def test_every_work_list_layout_keeps_results_exact(lb, monkeypatch, layout, rows):
    """Each layout (contiguous, packed, waves) and piece length, including
    pieces shorter than the stencil reach, gives each replica the result of
    the lattice run alone."""
    b = lb.Batch(8, lb.LB_F32)
    b.set_layout(layout, rows)
    slots = [b.add(nx, ny, _p(lb, ph, lb.LB_F32, bd, U), seed, steps)
             for nx, ny, ph, bd, U, seed, steps in REPLICAS]
    b.run(20)
    assert b.status() == lb.LB_OK
    for k, (nx, ny, ph, bd, U, seed, steps) in zip(slots, REPLICAS):
        ref = _alone(lb, monkeypatch, nx, ny, _p(lb, ph, lb.LB_F32, bd, U), seed, min(steps, 20))
        assert np.array_equal(b.get_state(k), ref), (nx, ny)
    b.close()
    with pytest.raises(lb.LBError):
        lb.Batch(2, lb.LB_F32).set_layout(3, 64)


def test_empty_and_spent_batches_run_as_no_ops(lb, monkeypatch):
    """A batch with no replicas, with every budget spent, or emptied by
    remove runs without error and leaves states untouched."""
    b = lb.Batch(3, lb.LB_F32)
    b.run(20)  # no replicas at all
    assert b.status() == lb.LB_OK
    p = _p(lb, CFG, lb.LB_F32, 0, 0.0)
    k = b.add(128, 32, p, 3, 0)  # no budget
    before = b.get_state(k)
    b.run(17)
    rem, done = b.poll()
    assert rem[k] == 0 and done[k] == 0
    assert np.array_equal(b.get_state(k), before)
    b.set_steps(k, 4)
    b.run(17)
    assert b.poll()[1][k] == 4
    assert np.array_equal(b.get_state(k), _alone(lb, monkeypatch, 128, 32, p, 3, 4))
    b.remove(k)
    b.run(16)
    assert b.status() == lb.LB_OK
    b.close()
