"""Pins of the oracle's time step, Eq. (be), against what the paper fixes.

* per-species mass and total momentum conserved to roundoff (periodic);
* a uniform state at rest is a fixed point;
* with all couplings off the scheme is D2Q9 BGK: a shear wave decays with
  nu = cs2 (tau - 1/2) (Sec. VI: nu = 1/6 at tau = 1);
* Couette walls (G = 0): the steady profile is linear and the wall stress is
  rho nu 2U/ny; per-species mass is conserved exactly with walls.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))


def test_mass_and_momentum_conserved_periodic():
    f = oracle.init_state(24, 20, 3, oracle.INIT_UNIFORM_NOISE, [1.0, 1.0, 0.05])
    ob0 = oracle.observables(f, CFG)
    g, bad = oracle.step(f, CFG, 60)
    ob1 = oracle.observables(g, CFG)
    assert bad == 0
    assert np.allclose(ob1["mass"][:2], ob0["mass"][:2], rtol=1e-13, atol=0)
    # total bare momentum starts at zero and stays zero to roundoff
    assert np.max(np.abs(ob1["mass"][2:])) < 1e-11
    # the run is not trivial: densities have moved
    assert np.max(np.abs(ob1["rho"] - ob0["rho"])) > 1e-3


def test_mass_and_momentum_conserved_unequal_tau():
    p = dict(CFG, tau=(0.8, 1.3), Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
    f = oracle.init_state(16, 18, 9, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    ob0 = oracle.observables(f, p)
    g, bad = oracle.step(f, p, 20)
    ob1 = oracle.observables(g, p)
    assert bad == 0
    assert np.allclose(ob1["mass"][:2], ob0["mass"][:2], rtol=1e-13, atol=0)
    assert np.max(np.abs(ob1["mass"][2:])) < 1e-11


def test_uniform_state_is_a_fixed_point():
    nx, ny = 9, 7
    rho = np.empty((2, ny, nx))
    rho[0] = 0.93
    rho[1] = 1.07
    f = rho[:, None] * W9[None, :, None, None]
    g, _ = oracle.step(f, CFG, 25)
    assert np.allclose(g, f, rtol=1e-15, atol=0)


def _shear_wave_nu(tau, ny=64, nx=5, t1=200, t2=1000, rho=(1.0, 1.0)):
    """Decay rate / k^2 of a sine shear wave of a uniform mixture; `tau` is one
    value or a (tau_A, tau_B) pair."""
    k = 2 * math.pi / ny
    y = np.arange(ny)
    ux = 1e-3 * np.sin(k * y)
    cu = CX[None, :, None, None] * ux[None, None, :, None]
    usq = (ux ** 2)[None, None, :, None]
    f = (W9[None, :, None, None] * np.asarray(rho, dtype=float)[:, None, None, None]
         * np.ones((2, 1, ny, nx)) * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * usq))
    p = dict(tau=tuple(tau) if np.ndim(tau) else (tau, tau))
    g1, _ = oracle.step(f, p, t1)
    g2, _ = oracle.step(g1, p, t2 - t1)

    def amp(g):
        u = oracle.observables(g, p)["u"][0].mean(axis=1)
        return 2 * np.dot(u, np.sin(k * y)) / ny

    return -math.log(amp(g2) / amp(g1)) / (k * k * (t2 - t1))


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_shear_wave_decay_gives_bgk_viscosity(tau):
    nu = _shear_wave_nu(tau)
    expect = float(Fraction(1, 3)) * (tau - 0.5)
    if tau == GOLD["viscosity_tau1"]["tau"]:
        assert expect == pytest.approx(float(Fraction(GOLD["viscosity_tau1"]["nu"])))
    # O(k^2) lattice corrections at k = 2 pi/64
    assert nu == pytest.approx(expect, rel=3e-3)


@pytest.mark.parametrize("taus,rho", [((0.8, 1.3), (0.7, 0.3)), ((0.6, 1.6), (0.5, 0.5))])
def test_mixture_viscosity_follows_the_mass_weighted_tau(taus, rho):
    """Unequal relaxation times (Sec. III footnote): the mixture relaxes with
    tau_bar = (rho_A tau_A + rho_B tau_B) / rho, nu = (tau_bar - 1/2)/3, up to
    O(k^2) (the deviation falls 4x when ny doubles); the harmonic mean, the
    other plausible reading, is far off."""
    rA, rB = rho
    tau_bar = (rA * taus[0] + rB * taus[1]) / (rA + rB)
    nu_bar = (tau_bar - 0.5) / 3.0
    dev = [_shear_wave_nu(taus, ny=ny, t1=100, t2=400, rho=rho) / nu_bar - 1.0 for ny in (32, 64)]
    assert abs(dev[1]) < 6e-3
    assert dev[0] / dev[1] == pytest.approx(4.0, rel=0.05)
    tau_h = (rA + rB) / (rA / taus[0] + rB / taus[1])
    assert abs((tau_h - 0.5) / 3.0 / nu_bar - 1.0) > 10 * abs(dev[1])


def test_couette_without_couplings_is_linear_with_wall_stress():
    ny, nx, U = 16, 5, 0.01
    p = dict(tau=(1.0, 1.0), boundary=oracle.COUETTE, U_wall=U)
    f = np.ones((2, 1, ny, nx)) * W9[None, :, None, None]
    g, _ = oracle.step(f, p, 6000)
    ob = oracle.observables(g, p)
    ux = ob["u"][0]
    exact = U * (2 * np.arange(ny) + 1 - ny) / ny  # walls at -1/2 and ny-1/2 moving -U, +U
    assert np.max(np.abs(ux - exact[:, None])) < 1e-10
    assert np.max(np.abs(ob["u"][1])) < 1e-13
    nu = (1.0 - 0.5) / 3.0
    sigma = 2.0 * nu * 2 * U / ny  # total density 2
    assert ob["stress"] == pytest.approx([sigma, sigma, sigma], rel=1e-7)


def test_couette_conserves_species_mass_with_full_couplings():
    p = dict(CFG, boundary=oracle.COUETTE, U_wall=0.05)
    f = oracle.init_state(20, 16, 1, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    m0 = oracle.observables(f, p)["mass"]
    g, bad = oracle.step(f, p, 50)
    m1 = oracle.observables(g, p)["mass"]
    assert bad == 0
    assert np.allclose(m1[:2], m0[:2], rtol=1e-13, atol=0)
    # the walls drive the fluid: x-momentum is no longer zero
    assert abs(m1[2]) > 1e-6


def test_couette_at_rest_is_a_fixed_point():
    nx, ny = 8, 9
    rho = np.empty((2, ny, nx))
    rho[0] = 0.8
    rho[1] = 1.2
    f = rho[:, None] * W9[None, :, None, None]
    p = dict(CFG, boundary=oracle.COUETTE, U_wall=0.0)
    g, _ = oracle.step(f, p, 20)
    assert np.allclose(g, f, rtol=1e-15, atol=0)
