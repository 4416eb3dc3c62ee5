"""Pins of the oracle's Kolmogorov shear (Sec. VII) and its diagnostics.

* With no couplings the body force g sin(ky) drives the Kolmogorov flow.  The
  steady common velocity plus half the force per mass, U_k + g/2, tends to
  the continuum amplitude g / (nu k^2) with nu = (tau - 1/2)/3 (Sec. VI): at
  tau = 1 with an error of fourth order in k (it falls 16x when ny doubles),
  for other tau of second order (4x).  The steady profile is a pure sine.
* U_k of a prescribed equilibrium state with u_x = A sin(ky) is A.
* I_AB (Eq. (INDICATOR)) equals a direct numpy evaluation with central
  differences (periodic, and mirrored rows at Couette walls).
"""
import numpy as np
import pytest

import inputs
import oracle

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _kolmogorov(ny, tau, g=1e-6, decay=20.0):
    p = dict(tau=(tau, tau), rho0=1.0, G_AB=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0), g_kolmo=g,
             k_kolmo=1)
    f = np.ones((2, 1, ny, 4)) * W9[None, :, None, None]
    nu, k = (tau - 0.5) / 3.0, 2.0 * np.pi / ny
    g_state, bad = oracle.step(f, p, int(decay / (nu * k * k)))  # transient e^-decay
    assert bad == 0
    return oracle.shear_diagnostics(g_state, p)["U_k"], g / (nu * k * k), g_state, p


def test_kolmogorov_flow_at_tau_one_converges_at_fourth_order():
    err = []
    for ny in (16, 32):
        uk, u0, _, _ = _kolmogorov(ny, 1.0)
        err.append((uk + 0.5e-6) / u0 - 1.0)
    assert abs(err[1]) < 1e-5
    assert err[0] / err[1] == pytest.approx(16.0, rel=0.1)


def test_kolmogorov_flow_converges_at_second_order():
    d32 = _kolmogorov(32, 0.8, decay=16.0)
    d64 = _kolmogorov(64, 0.8, decay=16.0)
    e32 = (d32[0] + 0.5e-6) / d32[1] - 1.0
    e64 = (d64[0] + 0.5e-6) / d64[1] - 1.0
    assert abs(e32) > 1e-4  # a real lattice correction at tau != 1 ...
    assert e32 / e64 == pytest.approx(4.0, rel=0.1)  # ... of second order in k


def test_kolmogorov_profile_is_a_pure_sine():
    uk, _, g_state, p = _kolmogorov(32, 0.8, decay=16.0)
    ux = oracle.observables(g_state, p)["u"][0]
    y = np.arange(32)
    assert np.max(np.abs(ux - uk * np.sin(2 * np.pi * y / 32)[:, None])) < 1e-11 * abs(uk)
    assert np.max(np.abs(oracle.observables(g_state, p)["u"][1])) < 1e-13


def _equilibrium(rho, ux, uy):
    cu = CX[:, None, None] * ux[None] + CY[:, None, None] * uy[None]
    usq = ux * ux + uy * uy
    return W9[:, None, None] * rho[None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq[None])


@pytest.mark.parametrize("k", [1, 3])
def test_u_k_of_a_prescribed_sine_flow(k):
    ny, nx, A = 48, 8, 0.013
    y = np.arange(ny)
    ux = np.tile((A * np.sin(2 * np.pi * k * y / ny))[:, None], (1, nx))
    uy = np.zeros_like(ux)
    rho = np.ones((ny, nx))
    f = np.stack([_equilibrium(rho, ux, uy), _equilibrium(rho, ux, uy)])
    d = oracle.shear_diagnostics(f, dict(tau=(1.0, 1.0), k_kolmo=k))
    assert d["U_k"] == pytest.approx(A, rel=1e-13)
    assert d["I_AB"] == pytest.approx(0.0, abs=1e-25)


@pytest.mark.parametrize("boundary", [0, 1])
def test_interface_indicator_matches_central_differences(boundary):
    ny, nx = 13, 11
    f = inputs.populations(nx, ny, seed=7, base=W9, rel_amp=0.3, species_scale=(0.8, 1.3))
    rho = f.sum(axis=1)  # [2][ny][nx]
    if boundary:  # mirrored rows about the walls: row -1 reads 0, row ny reads ny-1
        up = np.concatenate([rho[:, 1:], rho[:, -1:]], axis=1)
        dn = np.concatenate([rho[:, :1], rho[:, :-1]], axis=1)
    else:
        up, dn = np.roll(rho, -1, axis=1), np.roll(rho, 1, axis=1)
    gx = 0.5 * (np.roll(rho, -1, axis=2) - np.roll(rho, 1, axis=2))
    gy = 0.5 * (up - dn)
    expect = -np.sum(gx[0] * gx[1] + gy[0] * gy[1])
    d = oracle.shear_diagnostics(f, dict(tau=(1.0, 1.0), boundary=boundary))
    assert d["I_AB"] == pytest.approx(expect, rel=1e-13)
    assert d["I_AB"] != 0.0
