"""Pins of the oracle against the paper's equilibrium and transport theory.

The oracle is run to equilibrium on flat interfaces and droplets and compared
with the closed forms / root-finders of oracle/theory.py:
* pure repulsion: the zero-diffusion manifold rho_A/rho_B = exp((rho_A-rho_B)/rho_g^(tau))
  (Eq. (RHOGTAU), system (FIXING)) and the bulk densities (Sec. IV.A, Fig. 3);
* self-interactions: the symmetric bulk free energy (BULKfinal) (Sec. IV.C, Fig. 4);
* Laplace law P_in - P_out = sigma/R against sigma of (sigmaAB) with its tau terms,
  across tau at fixed rho_g^(tau) (Sec. V, Fig. 5);
* the vanishing-surface-tension crossover of Eq. (surften) (Fig. 6), and the
  simulated one of Fig. 7: sigma of (sigmaAB), with its tau terms, on
  equilibrated flat interfaces changes sign near the paper's rho0 = 0.717.
The paper states the agreement only qualitatively; tolerances are a few percent.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import theory as T

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _flat_interface(mean, p, nx=64, ny=5, steps=20000, hi=0.8):
    x = np.arange(nx)
    rA = np.where((x >= nx // 4) & (x < 3 * nx // 4), hi * mean, (1.0 - hi) * mean)
    rho = np.stack([np.tile(rA, (ny, 1)), np.tile(mean - rA, (ny, 1))])
    f = rho[:, None] * W9[None, :, None, None]
    g, bad = oracle.step(f, p, steps)
    assert bad == 0
    return oracle.densities(g)


def test_rho_g_of_the_paper():
    e1 = GOLD["E1_rho_g"]
    assert T.rho_g(e1["tau"], e1["g_AB"]) == pytest.approx(e1["rho_g"], abs=1e-5)


def test_taylor_closed_form_close_to_exact_roots():
    rh, rl = T.fixing_roots(3.5, 1.6)
    th, tl = T.taylor_roots(3.5, 1.6)
    assert rh + rl == pytest.approx(3.5)
    assert th == pytest.approx(rh, rel=1e-3) and tl == pytest.approx(rl, rel=1e-3)
    assert math.log(rh / rl) == pytest.approx((rh - rl) / 1.6, rel=1e-12)


@pytest.mark.slow
def test_pure_repulsion_flat_interface_matches_fixing():
    e1 = GOLD["E1_rho_g"]
    tau, g = e1["tau"], e1["g_AB"]
    rg = T.rho_g(tau, g)
    mean = 3.5
    p = dict(tau=(tau, tau), rho0=e1["rho0"], G_AB=g * e1["rho0"] ** 2)
    r = _flat_interface(mean, p)
    a, b = r[0, 2, 32], r[1, 2, 32]  # bulk of the A-rich slab
    # zero-diffusion manifold of (FIXING) holds in the bulk
    assert math.log(a / b) == pytest.approx((a - b) / rg, rel=1e-2)
    # bulk densities against the (FIXING) roots with <rho> as the bulk total
    rh, rl = T.fixing_roots(mean, rg)
    assert abs(a - rh) < 0.03 * mean and abs(b - rl) < 0.03 * mean
    # the B-rich slab mirrors it
    assert r[1, 2, 2] == pytest.approx(a, rel=1e-3) and r[0, 2, 2] == pytest.approx(b, rel=1e-3)


@pytest.mark.slow
def test_self_interaction_flat_interface_matches_bulkfinal_caption_set():
    """Fig. 4 caption set (tau = 1, g_AB = 0.5785, G1 = -0.63, F^r = 0)."""
    c = GOLD["fig4_caption"]
    p = dict(tau=(c["tau"], c["tau"]), rho0=c["rho0"], G_AB=c["g_AB"] * c["rho0"] ** 2,
             Ga=(c["G1_inset"], c["G1_inset"]), Gr=(0.0, 0.0))
    r = _flat_interface(c["mean_rho"], p)
    a, b = r[0, 2, 32], r[1, 2, 32]
    rh, rl = T.bulk_self_roots(c["mean_rho"], c["tau"], c["g_AB"], c["G1_inset"], c["rho0"])
    assert abs(a - rh) < 0.03 * c["mean_rho"] and abs(b - rl) < 0.03 * c["mean_rho"]
    # the text's set (tau = 0.69, g = 0.345) gives a clearly different theory value
    t = GOLD["fig4_text"]
    th_, tl_ = T.bulk_self_roots(t["mean_rho"], t["tau"], t["g_AB"], c["G1_inset"], t["rho0"])
    assert abs(tl_ - rl) > 0.1


@pytest.mark.slow
def test_self_interaction_config_couplings():
    """Both belts on (Ga = -9, Gr = 8.1, rho0 = 0.7): G1 = Ga + Gr enters the bulk."""
    p = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
    mean = 1.224
    r = _flat_interface(mean, p)
    a, b = r[0, 2, 32], r[1, 2, 32]
    G1, _ = T.effective_couplings(-9.0, 8.1)
    rh, rl = T.bulk_self_roots(mean, 1.0, 0.405 / 0.49, G1, 0.7)
    assert abs(a - rh) < 0.03 * mean and abs(b - rl) < 0.03 * mean


@pytest.mark.slow
def laplace_and_flat_sigma(tau, mean=2.5, n=64, R0=16, flat_steps=20000, drop_steps=8000):
    """Fig. 5 set-up (pure repulsion at fixed rho_g^(tau)): sigma of (sigmaAB) of a
    flat interface with and without its tau terms, and Delta p R of a droplet."""
    rg = GOLD["fig5_rho_g"]["rho_g"]
    g = T.theta(tau) / rg
    p = dict(tau=(tau, tau), rho0=1.0, G_AB=g)
    r = _flat_interface(mean, p, nx=64, ny=4, steps=flat_steps)
    sig_tau = T.sigma_flat_profile(r[0, 2], r[1, 2], tau, g, 0.0, 0.0, 1.0, slice(0, 32), True)
    sig_bare = T.sigma_flat_profile(r[0, 2], r[1, 2], tau, g, 0.0, 0.0, 1.0, slice(0, 32), False)
    yy, xx = np.mgrid[0:n, 0:n]
    d = np.sqrt((xx - n / 2 + 0.5) ** 2 + (yy - n / 2 + 0.5) ** 2)
    rA = np.where(d < R0, 0.8 * mean, 0.2 * mean)
    f = np.stack([rA, mean - rA])[:, None] * W9[None, :, None, None]
    gd, _ = oracle.step(f, p, drop_steps)
    rd = oracle.densities(gd)
    return sig_tau, sig_bare, laplace_of(rd, g)


def laplace_of(rd, g):
    """Delta p R of an equilibrated droplet: bulk pressures (PBULKINT) at the
    centre and in a corner, R from the A excess."""
    n = rd.shape[1]
    ain, aout = rd[0, n // 2, n // 2], rd[0, 2, 2]
    R = math.sqrt(((rd[0] - aout) / (ain - aout)).sum() / math.pi)
    dp = (T.bulk_pressure(rd[0, n // 2, n // 2], rd[1, n // 2, n // 2], g, 0, 0, 1.0)
          - T.bulk_pressure(rd[0, 2, 2], rd[1, 2, 2], g, 0, 0, 1.0))
    return dp * R


def test_laplace_law_needs_the_tau_corrections_fig5():
    """Fig. 5: at fixed rho_g^(tau) = 0.91, Delta p R of droplets follows sigma
    of (sigmaAB) with its tau terms (within 15 %, as at tau = 1) for every tau,
    while the bare sigma falls ever further behind as tau grows."""
    bare_err = []
    for tau in (0.7, 1.0, 1.5):
        sig_tau, sig_bare, lap = laplace_and_flat_sigma(tau)
        assert lap == pytest.approx(sig_tau, rel=0.15), tau
        assert abs(lap - sig_tau) < abs(lap - sig_bare), tau
        bare_err.append(abs(lap / sig_bare - 1.0))
    assert bare_err[0] < bare_err[1] < bare_err[2]
    assert bare_err[2] > 1.0  # at tau = 1.5 the bare sigma is off by more than 100 %


def test_effective_couplings_reproduce_printed_values():
    s = GOLD["standard_set_rho0_0_7"]
    f6 = GOLD["fig6_effective"]
    _, GA2 = T.effective_couplings(s["Ga"][0], s["Gr"][0])
    _, GB2 = T.effective_couplings(s["Ga"][1], s["Gr"][1])
    assert GA2 == pytest.approx(f6["G_A2"], abs=1e-4)
    assert GB2 == pytest.approx(f6["G_B2"], abs=1e-5)


def test_vanishing_surface_tension_crossover():
    f6 = GOLD["fig6_effective"]
    r0 = T.sigma_AB_crossover(f6["mean_rho"], f6["G_AB"], f6["G_A2"], f6["G_B2"])
    assert round(r0, f6["crossover_digits"]) == pytest.approx(f6["crossover_rho0"])
    # Sigma is positive below the crossover (repulsion wins) and negative above
    assert T.sigma_AB_criterion(r0 - 0.05, f6["mean_rho"], f6["G_AB"], f6["G_A2"], f6["G_B2"]) > 0
    assert T.sigma_AB_criterion(r0 + 0.05, f6["mean_rho"], f6["G_AB"], f6["G_A2"], f6["G_B2"]) < 0


def _sigma_of_flat_interface(rho0, steps=20000, nx=64):
    """sigma of (sigmaAB) with the tau terms, over one interface of a flat
    A-rich slab at <rho> = 1.23 with the rho0 = 0.7 standard couplings."""
    c = GOLD["fig7_simulated"]
    p = dict(tau=(c["tau"], c["tau"]), rho0=rho0, G_AB=c["G_AB"], Ga=tuple(c["Ga"]),
             Gr=tuple(c["Gr"]))
    # (a slab started near its bulk densities: from 0.8/0.2 it splits into lamellae)
    r = _flat_interface(c["mean_rho"], p, nx=nx, ny=4, steps=steps, hi=0.9)
    phi = r[0, 1] - r[1, 1]
    assert np.count_nonzero(np.sign(phi) != np.sign(np.roll(phi, 1))) == 2  # two interfaces
    _, GA2 = T.effective_couplings(c["Ga"][0], c["Gr"][0])
    _, GB2 = T.effective_couplings(c["Ga"][1], c["Gr"][1])
    return T.sigma_flat_profile(r[0, 1], r[1, 1], c["tau"], c["G_AB"], GA2, GB2, rho0,
                                slice(0, nx // 2), True)


def test_simulated_surface_tension_crossover_fig7():
    """Fig. 7: the simulated sigma(rho0) turns negative near rho0 = 0.717
    (0.71 in the caption); the theory of Eq. (surften) puts it at 0.7196.  The
    oracle's flat interfaces put it at 0.730: within 0.02 of all three (the
    paper's own values spread over 0.01, and neither the estimator behind
    Fig. 7 nor its lattice is stated)."""
    c = GOLD["fig7_simulated"]
    rho0s = (0.71, 0.75)
    sig = [_sigma_of_flat_interface(r) for r in rho0s]
    assert sig[0] > 0.0 > sig[1]  # repulsion wins below, self-interactions above
    x = T.zero_crossing(rho0s, sig)
    assert abs(x - c["crossover_rho0_text"]) < 0.02
    assert abs(x - c["crossover_rho0_caption"]) < 0.025
    f6 = GOLD["fig6_effective"]
    assert abs(x - T.sigma_AB_crossover(f6["mean_rho"], f6["G_AB"], f6["G_A2"], f6["G_B2"])) < 0.02
