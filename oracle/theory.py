"""Closed forms and root-finders of the paper's equilibrium and transport theory.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Each function restates one
result of Benzi et al., arXiv:0906.3611 (Secs. III-V); the tests use them as
pins for the FP64 oracle and, through it, for the CUDA path.

Readings of garbled passages (listed in the design notes as well):
  * (TAYLORRES) labels the "+" root as the low density; it is the high one.
  * The phi-form of the bulk free energy prints the interaction term as
    -(cs2/4) g (rho^2 - phi^2); with rho_A rho_B = (rho^2 - phi^2)/4 the
    sign is +, which is what gives the double well for rho > 2 rho_g.
  * (EQPSEUDO3) has cs2/2 where (P2) has cs2^2/2; the cs2^2 form is used,
    consistent with (sigmaAB).
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def theta(tau: float) -> float:
    """theta(tau) = (tau - 1/2)/tau, Eq. (THETA)."""
    return (tau - 0.5) / tau


def rho_g(tau: float, g_AB: float) -> float:
    """rho_g^(tau) = theta(tau)/g_AB, Eq. (RHOGTAU)."""
    return theta(tau) / g_AB


def effective_couplings(Ga: float, Gr: float):
    """(G_s1, G_s2) = (Ga + Gr, Ga + 12/7 Gr), Eq. (EFFECTIVE)."""
    return Ga + Gr, Ga + 12.0 / 7.0 * Gr


def _bisect(fun, lo: float, hi: float, tol: float = 1e-14, maxit: int = 400) -> float:
    flo = fun(lo)
    fhi = fun(hi)
    if flo == 0.0:
        return lo
    if fhi == 0.0:
        return hi
    if flo * fhi > 0:
        raise ValueError("root not bracketed")
    for _ in range(maxit):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if fm == 0.0 or (hi - lo) < tol * max(1.0, abs(mid)):
            return mid
        if flo * fm < 0:
            hi, fhi = mid, fm
        else:
            lo, flo = mid, fm
    return 0.5 * (lo + hi)


def fixing_roots(mean_rho: float, rg: float):
    """Bulk densities (rho_h, rho_l) of pure repulsion, system (FIXING):
    rho_A/rho_B = exp((rho_A - rho_B)/rho_g), rho_A + rho_B = <rho>.

    With phi = rho_A - rho_B the first line reads
    log((<rho> + phi)/(<rho> - phi)) = phi/rho_g; a non-trivial root exists
    only for <rho> > 2 rho_g.  Returns None below that threshold.
    """
    if mean_rho <= 2.0 * rg:
        return None

    def g(phi):
        return math.log((mean_rho + phi) / (mean_rho - phi)) - phi / rg

    eps = 1e-12 * mean_rho
    phi = _bisect(g, eps * 1e3, mean_rho * (1.0 - 1e-15))
    return 0.5 * (mean_rho + phi), 0.5 * (mean_rho - phi)


def taylor_roots(mean_rho: float, rg: float):
    """Closed-form approximation (TAYLORRES) of the (FIXING) roots.

    Returns (rho_h, rho_l); the paper's labels are swapped (see module doc).
    """
    inner = 45.0 * rg * rg - 10.0 * rg * mean_rho
    phi = math.sqrt(30.0 * rg * rg - 6.0 * rg * math.sqrt(inner))
    return 0.5 * (mean_rho + phi), 0.5 * (mean_rho - phi)


def psi(rho, rho0: float):
    """psi(rho) = rho0 (1 - exp(-rho/rho0)), Eq. (PSI)."""
    return rho0 * (1.0 - np.exp(-np.asarray(rho, dtype=float) / rho0))


def psi_sq_over_xi_sq_integral(rho: float, rho0: float, order: int = 200) -> float:
    """int_0^rho psi(xi)^2 / xi^2 dxi (the self-interaction term of (FREETOTAL)).

    The integrand is smooth on [0, rho] (it tends to 1 at xi -> 0), so plain
    Gauss-Legendre quadrature of high order is exact to roundoff.
    """
    x, w = np.polynomial.legendre.leggauss(order)
    xi = 0.5 * rho * (x + 1.0)
    val = (psi(xi, rho0) / xi) ** 2
    return float(0.5 * rho * np.dot(w, val))


def _h(rho: float, rho0: float) -> float:
    """d/drho [rho * int_0^rho psi^2/xi^2] = int_0^rho psi^2/xi^2 + psi(rho)^2/rho."""
    return psi_sq_over_xi_sq_integral(rho, rho0) + float(psi(rho, rho0)) ** 2 / rho


def bulk_self_roots(mean_rho: float, tau: float, g_AB: float, G1: float, rho0: float):
    """Symmetric bulk densities with self-interactions, Eq. (BULKfinal).

    f_b^(tau) = cs2 rho_A log rho_A + cs2 rho_B log rho_B + cs2 g^(tau) rho_A rho_B
              + cs2 G1^(tau)/2 [rho_A I(rho_A) + rho_B I(rho_B)],
    I(rho) = int_0^rho psi^2/xi^2, g^(tau) = g/theta, G1^(tau) = G1/theta.
    In the symmetric case the two phases are (rho_h, rho_l) and (rho_l, rho_h)
    and equilibrium needs d f_b/d rho_A = d f_b/d rho_B at (rho_h, rho_l):
      log(rho_h/rho_l) - g^(tau)(rho_h - rho_l) + G1^(tau)/2 [h(rho_h) - h(rho_l)] = 0
    with rho_h + rho_l = <rho>.  Returns (rho_h, rho_l) or None (no split).
    """
    th = theta(tau)
    gt = g_AB / th
    G1t = G1 / th

    def g(phi):
        rh = 0.5 * (mean_rho + phi)
        rl = 0.5 * (mean_rho - phi)
        return (math.log(rh / rl) - gt * (rh - rl)
                + 0.5 * G1t * (_h(rh, rho0) - _h(rl, rho0)))

    # the trivial root is phi = 0; bracket the non-trivial one by scanning
    grid = np.linspace(1e-6, 1.0 - 1e-9, 4001) * mean_rho
    vals = [g(p) for p in grid]
    for k in range(len(grid) - 1):
        if vals[k] < 0.0 <= vals[k + 1] or vals[k] > 0.0 >= vals[k + 1]:
            phi = _bisect(g, grid[k], grid[k + 1])
            return 0.5 * (mean_rho + phi), 0.5 * (mean_rho - phi)
    return None


def sigma_AB_criterion(rho0: float, mean_rho: float, G_AB: float, GA2: float, GB2: float) -> float:
    """Sigma_AB(rho0) = 2 G_AB/rho0^2 + 2/<rho> - (G_A2 + G_B2) exp(-<rho>/rho0), Eq. (surften)."""
    return 2.0 * G_AB / rho0 ** 2 + 2.0 / mean_rho - (GA2 + GB2) * math.exp(-mean_rho / rho0)


def sigma_AB_crossover(mean_rho: float, G_AB: float, GA2: float, GB2: float,
                       lo: float = 0.3, hi: float = 3.0) -> float:
    """The rho0 at which Sigma_AB(rho0) changes sign (vanishing surface tension)."""
    return _bisect(lambda r: sigma_AB_criterion(r, mean_rho, G_AB, GA2, GB2), lo, hi)


def bulk_pressure(rhoA, rhoB, g_AB: float, GA1: float, GB1: float, rho0: float):
    """Bulk part of P_ab, Eq. (PBULKINT) with Eq. (PBULKID):
    cs2 (rho_A + rho_B) + cs2 g rho_A rho_B + cs2/2 (G_A1 psi_A^2 + G_B1 psi_B^2)."""
    pA = psi(rhoA, rho0)
    pB = psi(rhoB, rho0)
    return (CS2 * (np.asarray(rhoA) + np.asarray(rhoB)) + CS2 * g_AB * np.asarray(rhoA) * np.asarray(rhoB)
            + 0.5 * CS2 * (GA1 * pA ** 2 + GB1 * pB ** 2))


def sigma_flat_profile(rhoA: np.ndarray, rhoB: np.ndarray, tau: float, G_AB: float,
                       GA2: float, GB2: float, rho0: float, window=None,
                       tau_terms: bool = True) -> float:
    """Surface tension of one flat interface from its density profiles, Eq. (sigmaAB).

    sigma = cs2^2 sum_x [ -G_A2/2 (d psi_A)^2 - G_B2/2 (d psi_B)^2 - G_AB/rho0^2 d rho_A d rho_B
                          + tau^2 theta^2 rho_A rho_B/rho (d rho_A/rho_A - d rho_B/rho_B)^2 ]
    The profiles are periodic; derivatives are centred differences on the
    whole profile and the sum runs over ``window`` (a slice holding exactly
    one interface; the whole profile if None).
    """
    rhoA = np.asarray(rhoA, dtype=float)
    rhoB = np.asarray(rhoB, dtype=float)
    dA = 0.5 * (np.roll(rhoA, -1) - np.roll(rhoA, 1))
    dB = 0.5 * (np.roll(rhoB, -1) - np.roll(rhoB, 1))
    pA = psi(rhoA, rho0)
    pB = psi(rhoB, rho0)
    dpA = 0.5 * (np.roll(pA, -1) - np.roll(pA, 1))
    dpB = 0.5 * (np.roll(pB, -1) - np.roll(pB, 1))
    integrand = -0.5 * GA2 * dpA ** 2 - 0.5 * GB2 * dpB ** 2 - G_AB / rho0 ** 2 * dA * dB
    if tau_terms:
        th = theta(tau)
        rho = rhoA + rhoB
        integrand = integrand + tau ** 2 * th ** 2 * rhoA * rhoB / rho * (dA / rhoA - dB / rhoB) ** 2
    if window is not None:
        integrand = integrand[window]
    return float(CS2 ** 2 * integrand.sum())


def zero_crossing(xs, ys) -> float:
    """x at which the sampled function y(x) first changes sign, by linear
    interpolation between the two bracketing samples (xs increasing)."""
    for k in range(len(xs) - 1):
        if ys[k] == 0.0:
            return float(xs[k])
        if ys[k] * ys[k + 1] < 0.0:
            return float(xs[k] - ys[k] * (xs[k + 1] - xs[k]) / (ys[k + 1] - ys[k]))
    raise ValueError("no sign change in the samples")
