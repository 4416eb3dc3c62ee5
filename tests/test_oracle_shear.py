"""Pins of the oracle's Kolmogorov shear (Sec. VII) and its diagnostics.

* With no couplings the body force g sin(ky) drives the Kolmogorov flow.  The
  steady common velocity plus half the force per mass, U_k + g/2, tends to
  the continuum amplitude g / (nu k^2) with nu = (tau - 1/2)/3 (Sec. VI): at
  tau = 1 with an error of fourth order in k (it falls 16x when ny doubles),
  for other tau of second order (4x).  The steady profile is a pure sine.
* U_k of a prescribed equilibrium state with u_x = A sin(ky) is A.
* I_AB (Eq. (INDICATOR)) takes closed-form values on fields whose central
  differences are known exactly: opposite ramps between Couette walls (the
  mirrored wall rows halve the difference there), opposite sine waves on a
  periodic lattice, and crossed gradients (zero).
* The ageing overlap (Eq. (CORRE)): C = cos(delta) for sine waves shifted by
  delta, a sign change under species exchange, C(t_w, 0) = 1, and the
  ensemble ratio of averaged sums.
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


def _state(rho_a, rho_b):
    """f = w_i rho_s at rest for density fields rho_s[ny, nx]."""
    return np.stack([W9[:, None, None] * rho_a[None], W9[:, None, None] * rho_b[None]])


def test_interface_indicator_of_opposite_ramps_between_walls():
    """rho_A = a + b y, rho_B = c - b y between Couette walls.  The central
    difference is b on interior rows and b/2 on the two wall rows (the stencil
    mirrors the density about each wall: row -1 reads row 0), so
    I_AB = -sum grad rho_A . grad rho_B = nx b^2 (ny - 2 + 2/4)."""
    nx, ny, a, b, c = 9, 14, 0.9, 0.02, 1.3
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    d = oracle.shear_diagnostics(_state(a + b * y, c - b * y), dict(tau=(1.0, 1.0), boundary=1))
    assert d["I_AB"] == pytest.approx(nx * b * b * (ny - 1.5), rel=1e-12)


@pytest.mark.parametrize("m", [1, 2])
def test_interface_indicator_of_opposite_sine_waves(m):
    """rho_A = a + e sin(kx), rho_B = c - e sin(kx), k = 2 pi m / nx, periodic:
    the central difference of sin(kx) is sin(k) cos(kx), so
    I_AB = e^2 sin(k)^2 sum cos^2(kx) = e^2 sin(k)^2 ny nx / 2."""
    nx, ny, a, c, e = 24, 7, 1.0, 0.8, 0.03
    k = 2.0 * np.pi * m / nx
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    d = oracle.shear_diagnostics(_state(a + e * np.sin(k * x), c - e * np.sin(k * x)),
                                 dict(tau=(1.0, 1.0), boundary=0))
    assert d["I_AB"] == pytest.approx(e * e * np.sin(k) ** 2 * ny * nx / 2.0, rel=1e-12)


def test_interface_indicator_of_crossed_gradients_vanishes():
    """A varying only along x and B only along y: the gradients are orthogonal
    at every site, so I_AB = 0 although both are nonzero (a transposed
    component in the dot product would not vanish)."""
    nx, ny = 16, 12
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    ra = 1.0 + 0.04 * np.sin(2 * np.pi * x / nx)
    rb = 0.7 + 0.05 * np.cos(2 * np.pi * y / ny)
    d = oracle.shear_diagnostics(_state(ra, rb), dict(tau=(1.0, 1.0), boundary=0))
    assert abs(d["I_AB"]) < 1e-15
    # the same fields with B varying along x instead: a nonzero closed form
    rb2 = 0.7 + 0.05 * np.sin(2 * np.pi * x / nx)
    d2 = oracle.shear_diagnostics(_state(ra, rb2), dict(tau=(1.0, 1.0), boundary=0))
    k = 2 * np.pi / nx
    assert d2["I_AB"] == pytest.approx(-0.04 * 0.05 * np.sin(k) ** 2 * ny * nx / 2, rel=1e-12)


# ---- ageing overlap, Eq. (CORRE) ----

def _phi_state(phi):
    """Densities 1 + phi/2 and 1 - phi/2: phi = rho_A - rho_B."""
    return _state(1.0 + 0.5 * phi, 1.0 - 0.5 * phi)


@pytest.mark.parametrize("delta", [0.0, np.pi / 3, np.pi / 2, np.pi])
def test_overlap_of_shifted_sine_waves(delta):
    """phi(t_w) = A sin(kx), phi(t) = A sin(kx + delta) on nx = one period:
    sum phi_w phi = A^2 ny (nx/2) cos(delta), sum phi_w^2 = A^2 ny nx/2, so
    C = cos(delta)."""
    nx, ny, A = 32, 5, 0.6
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    k = 2 * np.pi / nx
    num, den = oracle.phi_overlap(_phi_state(A * np.sin(k * x)), _phi_state(A * np.sin(k * x + delta)))
    assert den == pytest.approx(A * A * ny * nx / 2, rel=1e-12)
    assert num == pytest.approx(A * A * ny * nx / 2 * np.cos(delta), rel=1e-12, abs=1e-12)


def test_overlap_changes_sign_under_species_exchange():
    f_w = inputs.populations(10, 9, seed=3, base=W9, rel_amp=0.3, species_scale=(1.1, 0.6))
    f = inputs.populations(10, 9, seed=4, base=W9, rel_amp=0.3, species_scale=(0.9, 0.7))
    num, den = oracle.phi_overlap(f_w, f)
    num2, den2 = oracle.phi_overlap(f_w, f[::-1].copy())
    assert num2 == -num and den2 == den and num != 0.0
    assert oracle.phi_overlap(f_w, f_w) == (den, den)  # C(t_w, 0) = 1


def test_overlap_ensemble_averages_the_sums_not_the_ratios():
    """Eq. (CORRE) divides the ensemble averages of the two sums.  Realisation 1:
    A = 1, in phase (sums N/2, N/2); realisation 2: A = 3, in quadrature
    (0, 9N/2): C = (N/2) / (10 N/2) = 0.1, where the mean of the ratios is 0.5."""
    nx, ny = 16, 4
    x = np.ones((ny, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    k = 2 * np.pi / nx
    r1 = (_phi_state(np.sin(k * x)), _phi_state(np.sin(k * x)))
    r2 = (_phi_state(3 * np.sin(k * x)), _phi_state(3 * np.cos(k * x)))
    assert oracle.overlap_C([r1, r2]) == pytest.approx(0.1, rel=1e-12)
