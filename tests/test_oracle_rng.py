"""Pins of the oracle's seeded initial state.

* Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11);
* the two density recipes (uniform noise, Bernoulli droplet mixture) produce
  values in their stated ranges with the stated statistics, and f = w_i rho_s.
"""
import os

import numpy as np
import pytest

import oracle

KAT = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _kat_rows():
    rows = []
    for line in open(KAT):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox4x32_10(ctr, key) == out


def test_uniform_noise_recipe():
    rho = oracle.init_densities(64, 64, 0, oracle.INIT_UNIFORM_NOISE, [1.0, 1.0, 0.05])
    assert rho.min() >= 0.95 and rho.max() < 1.05
    assert abs(rho.mean() - 1.0) < 2e-3
    # uniform on [-0.05, 0.05): variance 0.05^2/3
    assert rho.var() == pytest.approx(0.05 ** 2 / 3, rel=0.05)
    assert abs(np.corrcoef(rho[0].ravel(), rho[1].ravel())[0, 1]) < 0.05


def test_bernoulli_recipe():
    rho = oracle.init_densities(64, 64, 0, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    hiA = rho[0] > 0.6
    assert abs(hiA.mean() - 0.7) < 0.03
    assert np.all(rho[1][hiA] < 0.6) and np.all(rho[1][~hiA] > 0.6)
    lo_ok = (rho >= 0.1) & (rho < 0.12)
    hi_ok = (rho >= 1.2) & (rho < 1.22)
    assert np.all(lo_ok | hi_ok)


def test_state_is_weighted_rest_state_and_seed_dependent():
    f = oracle.init_state(12, 10, 5, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    rho = oracle.init_densities(12, 10, 5, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    assert np.array_equal(f, rho[:, None] * W9[None, :, None, None])
    g = oracle.init_state(12, 10, 6, oracle.INIT_BERNOULLI, [0.7, 1.2, 0.1, 0.02])
    assert not np.array_equal(f, g)
