"""Pins of the oracle's response statistics (Sec. VIII, Figs. 14 and 16).

* Bursts planted at known steps in a quiet series are found exactly (starts,
  waits, log2 histogram), including runs of several steps.
* For a random walk with Gaussian steps the fraction of "above" steps is the
  Gaussian tail 2 (1 - Phi(c)), and the mean wait between burst starts is
  1 / (p (1 - p)) (starts of runs of a Bernoulli(p) sequence): this fixes mu,
  sigma (square root, population form) and the run logic.
* Log2 histogram of a hand-enumerated set of waits.
* Kurtosis: 3 for a Gaussian ensemble, 6 for a Laplace one, 1 for +-1.
* The power-law MLE recovers alpha = 2 from a sampled (rounded) power law.
"""
import math

import numpy as np
import pytest

import inputs
from oracle import response as RS


def test_planted_bursts_are_found_exactly():
    n = 5000
    rng = inputs.rng(3)
    d = 1e-6 * rng.standard_normal(n)
    runs = [(100, 1), (131, 3), (700, 2), (701 + 64, 1), (2000, 5), (4990, 1)]
    for s, length in runs:
        d[s:s + length] += 1.0
    U = np.concatenate([[0.25], 0.25 + np.cumsum(d)])
    r = RS.bursts(U, c=3.0, nbins=16)
    assert list(r["starts"]) == [s for s, _ in runs]
    assert list(r["waits"]) == [31, 569, 65, 1235, 2990]
    expect = np.zeros(16, dtype=np.int64)
    for b in (4, 9, 6, 10, 11):  # 31 -> [16,32), 569 -> [512,1024), 65, 1235, 2990
        expect[b] += 1
    assert np.array_equal(r["hist"], expect)
    assert r["events"] == len(runs)


def test_gaussian_walk_tail_fraction_and_mean_wait():
    n, c = 1_000_000, 2.0
    d = 0.01 * inputs.rng(5).standard_normal(n) + 0.003  # sigma != sigma^2, mu != 0
    U = np.concatenate([[0.0], np.cumsum(d)])
    dd = RS.derivative(U)
    mu, th = RS.threshold(dd, c)
    p = 2.0 * (1.0 - 0.5 * (1.0 + math.erf(c / math.sqrt(2.0))))  # 0.0455
    frac = float(np.mean(np.abs(dd - mu) > th))
    assert abs(frac - p) < 5.0 * math.sqrt(p * (1 - p) / n)
    w = RS.waiting_times(RS.burst_starts(U, c))
    assert float(np.mean(w)) == pytest.approx(1.0 / (p * (1.0 - p)), rel=0.03)


def test_log2_histogram_by_hand():
    w = [1, 2, 3, 4, 7, 8, 100]
    assert list(RS.log2_histogram(w, 8)) == [1, 2, 2, 1, 0, 0, 1, 0]
    assert list(RS.log2_histogram(w, 4)) == [1, 2, 2, 2]


def test_kurtosis_of_known_ensembles():
    rng = inputs.rng(9)
    assert RS.kurtosis(rng.standard_normal(400_000)) == pytest.approx(3.0, rel=0.02)
    assert RS.kurtosis(rng.laplace(size=400_000)) == pytest.approx(6.0, rel=0.04)
    assert RS.kurtosis(np.array([1.0, -1.0, 1.0, 1.0])) == 1.0


def test_powerlaw_mle_recovers_the_exponent():
    u = inputs.rng(11).uniform(size=200_000)
    x = np.rint(9.5 * u ** (-1.0 / (2.0 - 1.0)))  # continuous alpha = 2 above 9.5, rounded
    assert RS.powerlaw_alpha(x, 10) == pytest.approx(2.0, abs=0.02)
