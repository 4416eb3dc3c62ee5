"""N_s-species mixtures on the GPU (lb_mix_*, Sec. II: Eq. (be) and
Eq. (FORCE) for s = 1..N_s with a symmetric G_ss') against the FP64 oracle.

* FP64 one step from identical states: 1e-12 relative, for 2, 3 and 4
  species, periodic and Couette lattices spanning several tiles with ragged
  tails and the 5 x 5 minimum; 50 steps checked step by step.
* The seeded initial state is bit-identical to the oracle's recipe.
* FP32 one step: 1e-5 relative.
* Per-species mass and total momentum: FP64 reductions equal the oracle's
  observables of the same state, and are conserved by a free run.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
G3 = np.array([[0.0, 0.405, 0.21], [0.405, 0.0, 0.33], [0.21, 0.33, 0.0]])
MIX = {
    2: dict(ns=2, tau=[0.8, 1.3], rho0=0.83, Ga=[-9.0, -8.0], Gr=[8.1, 7.1],
            G=np.array([[0.0, 0.405], [0.405, 0.0]])),
    3: dict(ns=3, tau=[1.0, 0.9, 1.2], rho0=0.7, Ga=[-9.0, -8.5, -3.0], Gr=[8.1, 7.6, 2.5], G=G3),
    4: dict(ns=4, tau=[1.0, 0.9, 1.2, 0.7], rho0=0.7, Ga=[-9.0, -8.5, -3.0, 0.0],
            Gr=[8.1, 7.6, 2.5, 0.0],
            G=np.array([[0.0, 0.405, 0.21, 0.1], [0.405, 0.0, 0.33, 0.05],
                        [0.21, 0.33, 0.0, 0.02], [0.1, 0.05, 0.02, 0.0]])),
}


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _mix(lb, nx, ny, ns, storage, boundary=0, U=0.0):
    m = MIX[ns]
    p = lb.make_mix_params(m["ns"], m["tau"], m["rho0"], m["Ga"], m["Gr"], m["G"],
                           boundary=boundary, U_wall=U, storage=storage)
    return lb.Mixture(nx, ny, p)


def _op(ns, boundary=0, U=0.0):
    return dict(MIX[ns], boundary=boundary, U_wall=U)


def _state(ns, nx, ny, seed):
    scales = [0.9, 0.6, 0.3, 0.2][:ns]
    f = np.concatenate([inputs.populations(nx, ny, seed=seed + s, base=W9, rel_amp=0.05,
                                           species_scale=(scales[s], scales[s]))[:1]
                        for s in range(ns)])
    return f


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


SHAPES = [(64, 64), (67, 45), (5, 5), (131, 17)]


@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.03)])
@pytest.mark.parametrize("ns", [2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_one_step_parity(lb, shape, ns, boundary, U):
    nx, ny = shape
    f = _state(ns, nx, ny, seed=nx * 100 + ny)
    mx = _mix(lb, nx, ny, ns, lb.LB_F64, boundary, U)
    g = mx.set_state(f).step(1).get_state()
    assert mx.status() == lb.LB_OK
    mx.close()
    ref, bad = oracle.step_ns(f, _op(ns, boundary, U), 1)
    assert bad == 0
    assert _rel(g, ref) <= 1e-12


def test_seeded_init_is_bit_identical(lb):
    mean, amp = [0.8, 0.6, 0.3], [0.05, 0.05, 0.02]
    mx = _mix(lb, 70, 33, 3, lb.LB_F64)
    f = mx.init_random(77, mean, amp).get_state()
    mx.close()
    assert np.array_equal(f, oracle.init_ns(3, 70, 33, 77, mean, amp))


@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.02)])
def test_fp64_three_species_50_steps_step_by_step(lb, boundary, U):
    nx, ny = 96, 40
    f = oracle.init_ns(3, nx, ny, 5, [0.8, 0.6, 0.3], [0.05, 0.05, 0.02])
    mx = _mix(lb, nx, ny, 3, lb.LB_F64, boundary, U)
    worst = 0.0
    for t in range(50):
        nxt, bad = oracle.step_ns(f, _op(3, boundary, U), 1)
        assert bad == 0
        worst = max(worst, _rel(mx.set_state(f).step(1).get_state(), nxt))
        f = nxt
    mx.close()
    assert worst <= 1e-12


@pytest.mark.parametrize("ns", [2, 3])
def test_fp32_one_step(lb, ns):
    nx, ny = 133, 29
    f = _state(ns, nx, ny, seed=3).astype(np.float32).astype(np.float64)
    mx = _mix(lb, nx, ny, ns, lb.LB_F32, 1, 0.03)
    g = mx.set_state(f).step(1).get_state()
    mx.close()
    ref, _ = oracle.step_ns(f, _op(ns, 1, 0.03), 1)
    assert _rel(g, ref) <= 1e-5


def test_observables_match_the_oracle_and_are_conserved(lb):
    nx, ny = 128, 48
    mx = _mix(lb, nx, ny, 3, lb.LB_F64)
    mx.init_random(2, [0.8, 0.6, 0.3], [0.05, 0.05, 0.02])
    o0 = mx.observables()
    ref = oracle.observables_ns(mx.get_state(), _op(3))
    assert np.allclose(o0["mass"], ref["mass"], rtol=1e-13, atol=0)
    assert np.allclose(o0["momentum"], ref["momentum"], rtol=0, atol=1e-12)
    mx.step(500)
    o1 = mx.observables()
    assert mx.status() == lb.LB_OK
    mx.close()
    assert np.allclose(o1["mass"], o0["mass"], rtol=1e-13, atol=0)
    assert np.max(np.abs(o1["momentum"] - o0["momentum"])) < 1e-10


def test_fp32_mixture_mass_drift_is_a_random_walk(lb):
    """FP32 populations are stored as they are (no reference shift).  The
    rest population takes what the eight moving ones leave of rho_s, so a
    site's mass changes in a step only by roundings: the FP32 sums that form
    rho_s (8 additions, depth 4) and the eight stored values (depth 3), and
    the subtraction that forms the rest population -- about 15 roundings of
    values up to rho_s, each uniform within half an ulp (<= 2u rho_s, u =
    2^-24), so a standard deviation of at most sqrt(15 (2u)^2 / 12) ~ 2.2 u
    rho_s per site and step.  Unbiased and independent across N sites and
    T steps, the relative drift of a species' mass has a standard deviation of
    about 2.2 u sqrt(T / N); the bar is 10 u sqrt(T / N) (4.5 sd).  A biased
    collision breaks it: the nine equilibria summed in FP32 drifted by 1e-8
    per step (2e-5 here), the unfactored equilibrium with the mass-exact rest
    population by 3e-10 per step (6e-7 here, against the bar's 1e-7)."""
    G = np.array([[0.0, 0.405, 0.2], [0.405, 0.0, 0.2], [0.2, 0.2, 0.0]])
    p = lb.make_mix_params(3, [1.0, 1.0, 1.0], 0.7, [-9.0, -9.0, 0.0], [8.1, 8.1, 0.0], G,
                           boundary=0, U_wall=0.0, storage=lb.LB_F32)
    n, T = 256, 2000
    mx = lb.Mixture(n, n, p).init_random(7, [1.0, 1.0, 0.1], [0.05, 0.05, 0.01])
    m0 = mx.observables()["mass"][:3]
    mx.step(T)
    m1 = mx.observables()["mass"][:3]
    assert mx.status() == lb.LB_OK
    mx.close()
    bar = 10.0 * 2.0 ** -24 * np.sqrt(T / (n * n))
    assert float(np.max(np.abs(m1 / m0 - 1))) <= bar
