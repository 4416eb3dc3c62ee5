"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle.

This module only draws random numbers with numpy's counter-based Philox bit
generator and shapes them into arrays; it holds none of the lattice
Boltzmann arithmetic.  Callers pass any lattice-specific constants (such as a
base population vector) in.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def populations(nx: int, ny: int, seed: int, base, rel_amp: float = 0.05,
                species_scale=(1.0, 1.0)) -> np.ndarray:
    """f[2, 9, ny, nx] = species_scale[s] * base[i] * (1 + rel_amp * xi), xi ~ U(-1, 1).

    ``base`` is a length-9 positive vector supplied by the caller; independent
    noise on every population puts the state off any equilibrium manifold.
    """
    base = np.asarray(base, dtype=np.float64)
    xi = rng(seed).uniform(-1.0, 1.0, size=(2, 9, ny, nx))
    scale = np.asarray(species_scale, dtype=np.float64)[:, None, None, None]
    return scale * base[None, :, None, None] * (1.0 + rel_amp * xi)


def sample_sites(nx: int, ny: int, count: int, seed: int):
    """``count`` distinct (y, x) sites, always including the four corners."""
    g = rng(seed)
    pts = {(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)}
    while len(pts) < min(count, nx * ny):
        pts.add((int(g.integers(0, ny)), int(g.integers(0, nx))))
    return sorted(pts)


def fill_device_uniform(t, seed: int, lo: float, hi: float) -> None:
    """Fill a CUDA tensor in place with U(lo, hi) draws of torch's seeded
    Philox generator (for lattices too large to stage from the host)."""
    import torch
    g = torch.Generator(device=t.device)
    g.manual_seed(int(seed))
    t.uniform_(lo, hi, generator=g)
