"""Pins of the oracle's N_s-species step (Sec. II: Eq. (be) and Eq. (FORCE)
for species s = 1..N_s with a symmetric cross-coupling matrix G_ss').

* N_s = 2 reproduces the two-species passes bit for bit, and N_s = 3 with a
  third species of zero density and zero couplings reproduces them bit for
  bit on the first two species (the third stays empty).
* A single-site density spike of species 3 among uniform species gives, on
  species s at the sites whose first belt reaches it, the force
  -(G_s3 / rho0^2) rho_s w_j delta c_j and nothing elsewhere: the coupling
  matrix is indexed by the pair, not by the species alone.
* For symmetric G_ss' the forces sum to zero over the lattice, and per-species
  mass and total momentum are conserved to roundoff.
* Permuting the species (densities, tau, G^a, G^r and G consistently)
  permutes the result.
"""
import numpy as np
import pytest

import inputs
import oracle

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
ASYM2 = dict(tau=(0.8, 1.3), rho0=0.83, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
G3 = np.array([[0.0, 0.405, 0.21], [0.405, 0.0, 0.33], [0.21, 0.33, 0.0]])
MIX3 = dict(ns=3, tau=[1.0, 0.9, 1.2], rho0=0.7, Ga=[-9.0, -8.5, -3.0], Gr=[8.1, 7.6, 2.5], G=G3)


def _as_ns(p2: dict, ns: int) -> dict:
    """The two-species parameter dict as an ns-species one (extra species uncoupled)."""
    G = np.zeros((ns, ns))
    G[0, 1] = G[1, 0] = p2.get("G_AB", 0.0)
    pad = [1.0] * (ns - 2)
    zero = [0.0] * (ns - 2)
    return dict(ns=ns, tau=list(p2["tau"]) + pad, rho0=p2["rho0"], Ga=list(p2["Ga"]) + zero,
                Gr=list(p2["Gr"]) + zero, G=G, boundary=p2.get("boundary", 0),
                U_wall=p2.get("U_wall", 0.0), g_kolmo=p2.get("g_kolmo", 0.0),
                k_kolmo=p2.get("k_kolmo", 1))


@pytest.mark.parametrize("extra", [
    dict(), dict(boundary=1, U_wall=0.03), dict(g_kolmo=2e-4, k_kolmo=2)])
def test_two_species_reproduce_the_two_species_passes_bitwise(extra):
    p2 = dict(ASYM2, **extra)
    f = inputs.populations(23, 17, seed=3, base=W9, rel_amp=0.08, species_scale=(0.9, 1.1))
    ref, bad_ref = oracle.step(f, p2, 7)
    got, bad = oracle.step_ns(f, _as_ns(p2, 2), 7)
    assert np.array_equal(got, ref) and bad == bad_ref


@pytest.mark.parametrize("boundary", [0, 1])
def test_an_empty_uncoupled_third_species_changes_nothing(boundary):
    p2 = dict(ASYM2, boundary=boundary, U_wall=0.02)
    f = inputs.populations(19, 14, seed=5, base=W9, rel_amp=0.08, species_scale=(0.9, 1.1))
    f3 = np.concatenate([f, np.zeros((1, 9, 14, 19))])
    ref, _ = oracle.step(f, p2, 6)
    got, bad = oracle.step_ns(f3, _as_ns(p2, 3), 6)
    assert np.array_equal(got[:2], ref)
    assert np.all(got[2] == 0.0)
    assert bad == 6 * 14 * 19  # the empty species gets no velocity shift, and says so


def test_a_density_spike_of_species_3_pulls_on_each_species_through_its_own_coupling():
    n, rho0, delta = 9, 0.7, 0.05
    base = np.array([0.8, 0.6, 0.3])
    rho = base[:, None, None] * np.ones((3, n, n))
    y0, x0 = 4, 5
    rho[2, y0, x0] += delta
    p = dict(MIX3, Ga=[0.0, 0.0, -3.0], Gr=[0.0, 0.0, 2.5])  # only species 3 self-interacts
    F = oracle.forces_ns(rho, p)
    expect = np.zeros_like(F)
    for j in range(1, 9):  # belt 1: the site r0 - c_j sees r0 at offset c_j
        yy, xx = (y0 - CY[j]) % n, (x0 - CX[j]) % n
        for s in (0, 1):
            a = -(G3[s, 2] / rho0 ** 2) * rho[s, yy, xx] * W9[j] * delta
            expect[s, 0, yy, xx] += a * CX[j]
            expect[s, 1, yy, xx] += a * CY[j]
    assert np.allclose(F[:2], expect[:2], rtol=1e-12, atol=1e-17)
    assert np.max(np.abs(F[0])) > 0 and np.max(np.abs(F[1])) > 0
    # the two species feel the spike in the ratio of their couplings times densities
    k = (y0, (x0 - 1) % n)
    assert F[0, 0][k] / F[1, 0][k] == pytest.approx(G3[0, 2] * 0.8 / (G3[1, 2] * 0.6), rel=1e-12)


def test_forces_sum_to_zero_for_symmetric_couplings():
    rho = 0.5 + 0.3 * inputs.rng(8).uniform(0.0, 1.0, size=(3, 12, 15))
    F = oracle.forces_ns(rho, MIX3)
    scale = np.max(np.abs(F))
    assert np.max(np.abs(F.sum(axis=(0, 2, 3)))) < 1e-13 * scale * F[0, 0].size
    # an asymmetric matrix breaks the pairwise cancellation of F^X
    Gs = G3.copy()
    Gs[0, 2] = 0.5
    F2 = oracle.forces_ns(rho, dict(MIX3, G=Gs))
    assert np.max(np.abs(F2.sum(axis=(0, 2, 3)))) > 1e-6 * scale


def test_mass_of_every_species_and_total_momentum_are_conserved():
    f = oracle.init_ns(3, 32, 24, 11, [0.8, 0.6, 0.4], [0.05, 0.05, 0.05])
    o0 = oracle.observables_ns(f, MIX3)
    g, bad = oracle.step_ns(f, MIX3, 60)
    o1 = oracle.observables_ns(g, MIX3)
    assert bad == 0
    assert np.allclose(o1["mass"], o0["mass"], rtol=1e-13, atol=0)
    assert np.max(np.abs(o1["momentum"] - o0["momentum"])) < 1e-12
    assert np.max(np.abs(g - f)) > 1e-4  # the state did evolve


def test_a_species_permutation_permutes_the_result():
    f = oracle.init_ns(3, 20, 16, 4, [0.8, 0.6, 0.4], [0.05, 0.05, 0.05])
    perm = [2, 0, 1]
    pp = dict(MIX3, tau=[MIX3["tau"][k] for k in perm], Ga=[MIX3["Ga"][k] for k in perm],
              Gr=[MIX3["Gr"][k] for k in perm], G=G3[np.ix_(perm, perm)])
    a, _ = oracle.step_ns(f, MIX3, 10)
    b, _ = oracle.step_ns(f[perm], pp, 10)
    assert np.allclose(b, a[perm], rtol=1e-12, atol=1e-15)


def test_seeded_initial_state_follows_its_recipe():
    mean, amp = [0.8, 0.6, 0.4], [0.05, 0.02, 0.1]
    f = oracle.init_ns(3, 64, 64, 9, mean, amp)
    rho = f.sum(axis=1)
    for s in range(3):
        assert abs(rho[s].mean() - mean[s]) < 4 * amp[s] / np.sqrt(3 * 64 * 64)
        assert rho[s].min() >= mean[s] - amp[s] and rho[s].max() <= mean[s] + amp[s]
        assert np.std(rho[s]) == pytest.approx(amp[s] / np.sqrt(3), rel=0.05)
    assert np.allclose(f, W9[None, :, None, None] * rho[:, None], rtol=1e-15)
    # distinct species draw distinct numbers
    assert abs(np.corrcoef(rho[0].ravel(), rho[1].ravel())[0, 1]) < 0.05
