"""Pins of the oracle's pseudo-potential force, Eq. (FORCE) with Table I.

* a single-site density spike isolates every (direction, weight) pair of the
  24-speed stencil, with the weights taken from the paper's printed rationals;
* a brute-force 5x5 enumeration (weights looked up by |c|^2, not by index)
  on tiny periodic and wall-bounded lattices;
* uniform density gives zero force; the total force on a periodic lattice is
  zero (pairwise cancellation, so momentum is conserved);
* 90-degree rotations and reflections are equivariant; A<->B swap symmetry.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
P = {1: Fraction(GOLD["table_I_p"]["values"]["1-4"]), 2: Fraction(GOLD["table_I_p"]["values"]["5-8"]),
     4: Fraction(GOLD["table_I_p"]["values"]["9-12"]), 5: Fraction(GOLD["table_I_p"]["values"]["13-20"]),
     8: Fraction(GOLD["table_I_p"]["values"]["21-24"])}
W = {1: Fraction(GOLD["table_I_w"]["values"]["1-4"]), 2: Fraction(GOLD["table_I_w"]["values"]["5-8"])}

PRM = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))


def psi(r, rho0):
    return rho0 * (1.0 - math.exp(-r / rho0))


def test_uniform_density_gives_zero_force():
    rho = np.empty((2, 7, 9))
    rho[0] = 0.9
    rho[1] = 1.3
    F = oracle.forces(rho, PRM)
    assert np.max(np.abs(F)) < 1e-15


@pytest.mark.parametrize("species", [0, 1])
def test_single_site_spike_isolates_each_weight(species):
    """Spike delta in rho_s at r0: F_s(r0 - c_j) = -psi_u (Ga w_j + Gr p_j) dpsi c_j and
    F_s'(r0 - c_j) = -(G_AB/rho0^2) rho_s',u w_j drho c_j; zero everywhere else."""
    n = 11
    ru = (0.8, 1.1)
    drho = 0.07
    rho = np.empty((2, n, n))
    rho[0] = ru[0]
    rho[1] = ru[1]
    y0 = x0 = 5
    rho[species, y0, x0] += drho
    F = oracle.forces(rho, PRM)
    rho0 = PRM["rho0"]
    dpsi = psi(ru[species] + drho, rho0) - psi(ru[species], rho0)
    other = 1 - species
    Ga, Gr = PRM["Ga"][species], PRM["Gr"][species]
    g = PRM["G_AB"] / rho0 ** 2
    expect = np.zeros_like(F)
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            c2 = dx * dx + dy * dy
            if c2 == 0:
                continue
            yy, xx = y0 - dy, x0 - dx
            wj = float(W.get(c2, 0))
            pj = float(P[c2])
            coef_s = -psi(ru[species], rho0) * (Ga * wj + Gr * pj) * dpsi
            expect[species, 0, yy, xx] = coef_s * dx
            expect[species, 1, yy, xx] = coef_s * dy
            coef_o = -g * ru[other] * wj * drho
            expect[other, 0, yy, xx] = coef_o * dx
            expect[other, 1, yy, xx] = coef_o * dy
    assert np.allclose(F, expect, rtol=1e-12, atol=1e-15)


def _brute_force(rho, prm, couette):
    """Independent enumeration over the 5x5 square of offsets, weights by |c|^2."""
    _, ny, nx = rho.shape
    rho0 = prm["rho0"]
    g = prm["G_AB"] / rho0 ** 2
    ps = rho0 * (1.0 - np.exp(-rho / rho0))

    def row(y):
        if not couette:
            return y % ny
        if y < 0:
            return -1 - y
        if y >= ny:
            return 2 * ny - 1 - y
        return y

    F = np.zeros((2, 2, ny, nx))
    for s in range(2):
        o = 1 - s
        for y in range(ny):
            for x in range(nx):
                acc = np.zeros(2)
                for dy in range(-2, 3):
                    for dx in range(-2, 3):
                        c2 = dx * dx + dy * dy
                        if c2 == 0:
                            continue
                        yy, xx = row(y + dy), (x + dx) % nx
                        wgt = prm["Ga"][s] * float(W.get(c2, 0)) + prm["Gr"][s] * float(P[c2])
                        acc += -ps[s, y, x] * wgt * ps[s, yy, xx] * np.array([dx, dy])
                        acc += -g * rho[s, y, x] * float(W.get(c2, 0)) * rho[o, yy, xx] * np.array([dx, dy])
                F[s, :, y, x] = acc
    return F


@pytest.mark.parametrize("shape", [(5, 5), (6, 7), (5, 9)])
@pytest.mark.parametrize("couette", [False, True])
def test_brute_force_hand_sums(shape, couette):
    rng = np.random.default_rng(7 + shape[0] * 10 + shape[1] + 100 * couette)
    rho = rng.uniform(0.05, 1.5, size=(2,) + shape)
    prm = dict(PRM, boundary=oracle.COUETTE if couette else oracle.PERIODIC)
    F = oracle.forces(rho, prm)
    assert np.allclose(F, _brute_force(rho, PRM, couette), rtol=1e-12, atol=1e-14)


def test_total_force_vanishes_on_periodic_lattice():
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 1.4, size=(2, 12, 10))
    F = oracle.forces(rho, PRM)
    total = F.sum(axis=(2, 3)).sum(axis=0)
    assert np.max(np.abs(total)) < 1e-12


def _rotate90(a):
    """(x, y) -> (-y, x) on an n x n periodic lattice; a[y, x] indexing."""
    n = a.shape[-1]
    out = np.empty_like(a)
    for y in range(n):
        for x in range(n):
            out[..., x % n, (-y) % n] = a[..., y, x]
    return out


def test_rotation_and_reflection_equivariance():
    rng = np.random.default_rng(11)
    n = 8
    rho = rng.uniform(0.1, 1.4, size=(2, n, n))
    F = oracle.forces(rho, PRM)
    Fr = oracle.forces(_rotate90(rho), PRM)
    # rotated force field: F'(Rr) = R F(r) with R(x, y) = (-y, x)
    Fx_rot = _rotate90(-F[:, 1])
    Fy_rot = _rotate90(F[:, 0])
    assert np.allclose(Fr[:, 0], Fx_rot, atol=1e-14)
    assert np.allclose(Fr[:, 1], Fy_rot, atol=1e-14)
    # reflection x -> -x
    refl = rho[:, :, (-np.arange(n)) % n]
    Fm = oracle.forces(refl, PRM)
    assert np.allclose(Fm[:, 0], -F[:, 0][:, :, (-np.arange(n)) % n], atol=1e-14)
    assert np.allclose(Fm[:, 1], F[:, 1][:, :, (-np.arange(n)) % n], atol=1e-14)


def test_species_swap_symmetry():
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.1, 1.4, size=(2, 6, 9))
    sym = dict(PRM, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
    F = oracle.forces(rho, sym)
    Fs = oracle.forces(rho[::-1].copy(), sym)
    assert np.allclose(Fs, F[::-1], atol=1e-15)
