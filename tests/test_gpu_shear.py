"""Kolmogorov shear (Sec. VII) on the GPU, against the FP64 oracle.

* One step with the body force: FP64 1e-12 (both step kernels, periodic and
  Couette lattices, the paper's rho0 = 0.7 standard couplings), FP32 1e-5.
* Without couplings the GPU reaches the oracle's pinned Kolmogorov flow:
  U_k + g/2 = g / (nu k^2) to fourth order at tau = 1.
* lb_shear_diagnostics equals the oracle's diagnostics of the same state
  (U_k and I_AB to 1e-12 for FP64 storage).
* lb_phi_overlap equals the oracle's overlap sums (Eq. (CORRE)) to 1e-12.
* A batched replica with the body force equals the lattice run alone.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
# Eq. (STANDARD07): rho0 = 0.7, (Ga, Gr) = (-15, 14.1) for A and (-14, 13.1) for B
STD07 = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-15.0, -14.0), Gr=(14.1, 13.1))


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("kernel", ["rows", "tile"])
@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.02)])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_one_step_with_the_body_force(lb, monkeypatch, kernel, boundary, U, storage, tol):
    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", kernel)
    nx, ny, g, k = 264, 40, 2e-3, 3
    f = inputs.populations(nx, ny, seed=21, base=W9, rel_amp=0.05, species_scale=(0.6, 0.62))
    if storage == "f32":
        f = f.astype(np.float32).astype(np.float64)
    p = lb.make_params(**STD07, boundary=boundary, U_wall=U, storage=st, rho_ref=(0.6, 0.62),
                       g_kolmo=g, k_kolmo=k)
    lat = lb.Lattice(nx, ny, p)
    out = lat.set_state(f).step(1).get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, bad = oracle.step(f, dict(STD07, boundary=boundary, U_wall=U, g_kolmo=g, k_kolmo=k), 1)
    assert bad == 0
    assert _rel(out, ref) <= tol
    # the force mattered: without it the step differs by far more than the tolerance
    ref0, _ = oracle.step(f, dict(STD07, boundary=boundary, U_wall=U), 1)
    assert _rel(ref0, ref) > 100 * tol


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-5)])
def test_kolmogorov_flow_without_couplings(lb, storage, tol):
    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    ny, nx, g = 32, 128, 1e-6
    p = lb.make_params(tau=(1.0, 1.0), rho0=1.0, G_AB=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0),
                       storage=st, rho_ref=(1.0, 1.0), g_kolmo=g, k_kolmo=1)
    lat = lb.Lattice(nx, ny, p)
    lat.set_state(np.ones((2, 1, ny, nx)) * W9[None, :, None, None])
    nu, k = 0.5 / 3.0, 2 * np.pi / ny
    lat.step(int(20 / (nu * k * k)))
    uk = lat.shear_diagnostics()["U_k"]
    assert lat.status() == lb.LB_OK
    lat.close()
    # the oracle's pinned value at this size (fourth-order lattice error, 6.2e-6)
    ref = 6.2e-6
    assert (uk + g / 2) / (g / (nu * k * k)) - 1 == pytest.approx(ref, abs=max(tol, 2e-7))


@pytest.mark.parametrize("boundary", [0, 1])
def test_shear_diagnostics_match_the_oracle(lb, boundary):
    nx, ny = 136, 48
    pd = dict(STD07, boundary=boundary, U_wall=0.01 * boundary, g_kolmo=1e-4, k_kolmo=1)
    p = lb.make_params(**STD07, boundary=boundary, U_wall=0.01 * boundary, storage=lb.LB_F64,
                       rho_ref=(0.6, 0.6), init_kind=lb.LB_INIT_UNIFORM_NOISE,
                       init=(0.612, 0.612, 0.01), g_kolmo=1e-4, k_kolmo=1)
    lat = lb.Lattice(nx, ny, p).init_random(4).step(300)
    d = lat.shear_diagnostics()
    f = lat.get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref = oracle.shear_diagnostics(f, pd)
    assert ref["bad"] == 0
    assert d["U_k"] == pytest.approx(ref["U_k"], rel=1e-12)
    assert d["I_AB"] == pytest.approx(ref["I_AB"], rel=1e-12)
    assert abs(d["U_k"]) > 0 and d["I_AB"] > 0  # flowing; interfaces present


def test_batched_kolmogorov_replicas_equal_the_lattice_alone(lb, monkeypatch):
    p1 = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                        init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                        g_kolmo=2e-5, k_kolmo=1)
    p2 = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                        init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                        g_kolmo=6e-5, k_kolmo=2)
    b = lb.Batch(4, lb.LB_F32)
    s1 = b.add(128, 128, p1, 1, 40)
    s2 = b.add(256, 64, p2, 2, 40)
    b.run(40)
    assert b.status() == lb.LB_OK
    got = [b.get_state(s1), b.get_state(s2)]
    diag = [b.shear_diagnostics(s1), b.shear_diagnostics(s2)]
    b.close()
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    for (nx, ny, p, seed), g, d in zip([(128, 128, p1, 1), (256, 64, p2, 2)], got, diag):
        lat = lb.Lattice(nx, ny, p).init_random(seed).step(40)
        assert np.array_equal(lat.get_state(), g)
        assert lat.shear_diagnostics() == d
        lat.close()


def test_ageing_overlap_matches_the_oracle(lb):
    """Eq. (CORRE) sums of lb_phi_overlap against the oracle's on two states of
    an FP64 Kolmogorov-sheared trajectory that the oracle ran (t_w = 200 and
    t_w + 150 from the seeded start), to 1e-12 relative; the snapshot survives
    the state exchange, and C(t_w, 0) = 1."""
    nx, ny = 136, 48
    op = dict(STD07, g_kolmo=1e-4, k_kolmo=1)
    f0 = oracle.init_state(nx, ny, 8, oracle.INIT_UNIFORM_NOISE, (0.612, 0.612, 0.01))
    f_w, _ = oracle.step(f0, op, 200)
    f_t, _ = oracle.step(f_w, op, 150)
    num_ref, den_ref = oracle.phi_overlap(f_w, f_t)
    p = lb.make_params(**STD07, storage=lb.LB_F64, rho_ref=(0.6, 0.6),
                       init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                       g_kolmo=1e-4, k_kolmo=1)
    lat = lb.Lattice(nx, ny, p).init_random(8)
    assert np.array_equal(lat.get_state(), f0)
    with pytest.raises(lb.LBError):
        lat.phi_overlap()  # no snapshot yet
    lat.set_state(f_w).phi_snapshot()
    num0, den0 = lat.phi_overlap()
    assert num0 == den0  # C(t_w, 0) = 1
    assert den0 == pytest.approx(den_ref, rel=1e-12)
    lat.set_state(f_t)
    num, den = lat.phi_overlap()
    lat.close()
    assert den == pytest.approx(den_ref, rel=1e-12)
    assert num == pytest.approx(num_ref, rel=1e-12)
    assert 0.0 < num / den < 1.0  # the configuration has moved


def test_batched_overlap_equals_the_lattice_alone(lb, monkeypatch):
    p = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                       init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                       g_kolmo=2e-5, k_kolmo=1)
    b = lb.Batch(2, lb.LB_F32)
    s = b.add(128, 128, p, 5, 60)
    b.run(30)
    b.phi_snapshot(s)
    b.run(30)
    got = b.phi_overlap(s)
    b.close()
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    lat = lb.Lattice(128, 128, p).init_random(5).step(30).phi_snapshot().step(30)
    assert lat.phi_overlap() == got
    lat.close()


@pytest.mark.parametrize("kernel", ["rows", "tile"])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_series_records_the_response_of_every_step(lb, monkeypatch, kernel, storage, tol):
    """Entry t of the record is U_k of the state at the start of step t."""
    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", kernel)
    p = lb.make_params(**STD07, storage=st, rho_ref=(0.612, 0.612),
                       init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                       g_kolmo=5e-5, k_kolmo=2)
    lat = lb.Lattice(256, 96, p).init_random(3).step(10)
    lat.series_start(16)
    expect = []
    for _ in range(40):  # diagnostics of each state, then the step that records it
        expect.append(lat.shear_diagnostics()["U_k"])
        lat.step(1)
    got = lat.series()
    assert lat.status() == lb.LB_OK
    assert len(got) == 16  # the ring keeps the most recent 16 steps
    assert np.max(np.abs(got - np.array(expect[-16:]))) <= tol * np.max(np.abs(expect))
    lat.step(64)  # graph-replayed steps record too
    assert len(lat.series()) == 16
    lat.series_stop().step(3)
    with pytest.raises(lb.LBError):
        lat.series()
    lat.close()


def test_batch_with_forced_and_plain_replicas_coming_and_going(lb, monkeypatch):
    """Forced and unforced replicas share a launch; removing the forced one
    switches the batch back to the plain kernel variant mid-run."""
    common = dict(STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                  init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01))
    pf = lb.make_params(**common, g_kolmo=4e-5, k_kolmo=1)
    pp = lb.make_params(**common)
    b = lb.Batch(4, lb.LB_F32)
    sf = b.add(128, 128, pf, 1, 64)
    sp = b.add(160, 64, pp, 2, 64)
    b.run(32)  # two replayed 16-step graphs
    forced = b.get_state(sf)
    b.remove(sf)
    b.run(32)
    assert b.status() == lb.LB_OK
    plain = b.get_state(sp)
    b.close()
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    lat = lb.Lattice(128, 128, pf).init_random(1).step(32)
    assert np.array_equal(lat.get_state(), forced)
    lat.close()
    lat = lb.Lattice(160, 64, pp).init_random(2).step(64)
    assert np.array_equal(lat.get_state(), plain)
    lat.close()


def test_batched_series_equal_the_lattice_alone(lb, monkeypatch):
    """A replica's record equals the record of the same lattice run alone (the
    states are identical; each compute warp sums its sites in the arithmetic
    type, FP32 here, over the rows of its work item, and the batch cuts the
    rows differently: 1e-6 of the largest entry); replicas without a record
    and forced replicas without one run beside it; stopping ends the record."""
    pf = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                        init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                        g_kolmo=5e-5, k_kolmo=1)
    pp = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                        init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01))
    b = lb.Batch(4, lb.LB_F32)
    s1 = b.add(256, 128, pf, 1, 100)
    s2 = b.add(128, 128, pf, 2, 100)
    s3 = b.add(192, 64, pp, 3, 100)
    b.run(4)
    b.series_start(s1, 64).series_start(s3, 8)
    b.run(40)  # two replayed 16-step graphs and 8 single launches
    got1, got3 = b.series(s1), b.series(s3)
    b.series_stop(s3)
    b.run(3)
    with pytest.raises(lb.LBError):
        b.series(s3)
    assert len(b.series(s1)) == 43
    assert b.status() == lb.LB_OK
    b.close()
    assert len(got1) == 40 and len(got3) == 8
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    for (nx, ny, p, seed, cap), got in (((256, 128, pf, 1, 64), got1), ((192, 64, pp, 3, 8), got3)):
        lat = lb.Lattice(nx, ny, p).init_random(seed).step(4).series_start(cap).step(40)
        ref = lat.series()
        lat.close()
        assert len(ref) == len(got)
        assert np.max(np.abs(ref - got)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("c", [0.5, 1.0])
def test_burst_statistics_match_the_oracle(lb, c):
    """lb_series_bursts / lb_batch_series_bursts equal oracle.response.bursts of
    the same record, bit for bit: a wrapped ring of 4095 entries, four
    analysis chunks, bursts across chunk edges.  (FP16 storage: its
    stochastic rounding makes the recorded derivative jagged, so that there
    are many bursts to compare.)"""
    from oracle import response as RS
    p = lb.make_params(**STD07, storage=lb.LB_F16_DEV, rho_ref=(0.612, 0.612),
                       init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                       g_kolmo=2e-5, k_kolmo=1)
    lat = lb.Lattice(128, 128, p).init_random(7).series_start(4095).step(5000)
    U = lat.series()
    got = lat.series_bursts(c, 12)
    assert lat.status() == lb.LB_OK
    lat.close()
    assert len(U) == 4095
    ref = RS.bursts(U, c, 12)
    d = RS.derivative(U)
    mu, th = RS.threshold(d, c)
    assert np.min(np.abs(np.abs(d - mu) - th)) > 1e-9 * th  # no decision at the FP edge
    assert got["events"] == ref["events"] > 10
    assert np.array_equal(got["hist"], ref["hist"])
    # the same replica in a batch
    b = lb.Batch(2, lb.LB_F16_DEV)
    s = b.add(128, 128, p, 7, 5000)
    b.add(96, 64, p, 8, 5000)
    b.series_start(s, 4095)
    b.run(5000)
    Ub, gb = b.series(s), b.series_bursts(s, c, 12)
    b.close()
    rb = RS.bursts(Ub, c, 12)
    assert gb["events"] == rb["events"] and np.array_equal(gb["hist"], rb["hist"])


def test_burst_statistics_of_short_records(lb):
    p = lb.make_params(**STD07, storage=lb.LB_F32, rho_ref=(0.612, 0.612),
                       g_kolmo=2e-5, k_kolmo=1)
    lat = lb.Lattice(128, 64, p).init_random(1)
    with pytest.raises(lb.LBError):
        lat.series_bursts()  # no record
    lat.series_start(100)
    for steps in (0, 1, 2):  # fewer than two derivative samples: no bursts
        r = lat.series_bursts(2.0, 4)
        assert r["events"] == 0 and not r["hist"].any()
        lat.step(1)
    with pytest.raises(lb.LBError):
        lat.series_bursts(-1.0, 4)
    with pytest.raises(lb.LBError):
        lat.series_bursts(2.0, 65)
    lat.close()
