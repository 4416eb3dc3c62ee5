"""Response statistics of Sec. VIII from a recorded series (oracle).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the reference the
device analysis of a shear-response record is checked against.  Plain numpy,
FP64, in the order the quantities are defined.

* Bursts of dU/dt (Fig. 14).  The paper shows the time derivative of the
  response, its intermittent bursts ("events") and the pdf of the time lapse
  Delta t_e between subsequent bursts, decaying like Delta t_e^-2; it does not
  define a burst.  Reading: with d_j = U_{j+1} - U_j the one-step derivative,
  mu and sigma its mean and (population) standard deviation over the record,
  step j is "above" when |d_j - mu| > c sigma; a burst is a maximal run of
  consecutive above steps, it starts at the first step of the run, and the
  waiting times are the differences of successive burst starts.
* Waiting-time histogram: bin b counts waits in [2^b, 2^(b+1)) (the last bin
  also takes every longer wait).
* Kurtosis over an ensemble at fixed t (Fig. 16): <R^4> / <R^2>^2.
* Power-law exponent of the waits: the maximum-likelihood estimate for a
  continuous power law above x_min, alpha = 1 + n / sum ln(x_i / x_min)
  (Clauset, Shalizi and Newman, SIAM Review 51 (2009), Eq. 3.1), applied to
  waits >= x_min with x_min - 1/2 in the logarithm (their discrete
  approximation, Eq. 3.7).
"""
from __future__ import annotations

import math

import numpy as np


def derivative(U) -> np.ndarray:
    """d_j = U_{j+1} - U_j, j = 0 .. n-2."""
    U = np.asarray(U, dtype=np.float64)
    return U[1:] - U[:-1]


def threshold(d, c: float) -> tuple[float, float]:
    """(mu, c sigma) of the derivative samples d (population sigma)."""
    d = np.asarray(d, dtype=np.float64)
    mu = float(np.mean(d))
    sigma = math.sqrt(max(float(np.mean(d * d)) - mu * mu, 0.0))
    return mu, c * sigma


def burst_starts(U, c: float) -> np.ndarray:
    """Indices j (into d) where a run of |d_j - mu| > c sigma begins."""
    d = derivative(U)
    if d.size < 2:
        return np.zeros(0, dtype=np.int64)
    mu, th = threshold(d, c)
    above = np.abs(d - mu) > th
    prev = np.concatenate([[False], above[:-1]])
    return np.nonzero(above & ~prev)[0].astype(np.int64)


def waiting_times(starts) -> np.ndarray:
    """Differences of successive burst starts."""
    s = np.asarray(starts, dtype=np.int64)
    return s[1:] - s[:-1]


def log2_histogram(waits, nbins: int) -> np.ndarray:
    """Bin b counts waits w with 2^b <= w < 2^(b+1); the last bin takes the rest."""
    h = np.zeros(nbins, dtype=np.int64)
    for w in np.asarray(waits, dtype=np.int64):
        b = int(w).bit_length() - 1  # floor(log2 w) for w >= 1
        h[min(b, nbins - 1)] += 1
    return h


def bursts(U, c: float, nbins: int) -> dict:
    """Starts, waits and the log2 histogram of the waits of a series."""
    s = burst_starts(U, c)
    w = waiting_times(s)
    return {"starts": s, "waits": w, "hist": log2_histogram(w, nbins), "events": int(s.size)}


def kurtosis(R) -> float:
    """<R^4> / <R^2>^2 over the ensemble R (Fig. 16)."""
    R = np.asarray(R, dtype=np.float64)
    return float(np.mean(R ** 4) / np.mean(R ** 2) ** 2)


def powerlaw_alpha(waits, x_min: float) -> float:
    """Maximum-likelihood power-law exponent of the waits >= x_min."""
    w = np.asarray(waits, dtype=np.float64)
    w = w[w >= x_min]
    return 1.0 + w.size / float(np.sum(np.log(w / (x_min - 0.5))))
