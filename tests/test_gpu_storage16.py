"""Reduced-precision storage: FP32 arithmetic on populations stored as BF16 or
FP16 deviations d_i = f_i - w_i rho_ref,s, against the FP64 oracle.

* One step from a state near rho_ref, both step kernels, both boundary kinds:
  every population within a bound derived from the storage format, with no
  fitted factor.  The oracle steps the stored (rounded) state, so the GPU's
  error is (1) the FP32 arithmetic, held to the FP32 bar 1e-5 w_i rho_s;
  (2) the round-to-nearest of each stored moving deviation, at most
  u |d*_i| (u = 2^-11 FP16, 2^-8 BF16) plus half the smallest subnormal
  spacing; (3) for the rest population, which takes what the eight stored
  moving populations leave of the site's density deviation, the sum of those
  eight roundings plus its own stochastic rounding (under one unit in the
  last place, 2u |d*_0|).
* Per-species mass drift of the 512 x 512 Bernoulli droplet emulsion after
  1000 steps (rho_ref = the species means): FP32 <= 1e-6 (stated; measured
  1e-8); the 16-bit drift is a random walk of one stochastic rounding per site
  and step, of at most one unit in the last place of |d_0| <= 4/9 |rho -
  rho_ref| <= 0.35 (variance <= ulp^2/6), so its relative standard deviation is
  ulp sqrt(T / (6 N)) / <rho_s> and the bound four of those (FP16 ulp 2^-12:
  5.7e-5, BF16 ulp 2^-9: 4.6e-4 with <rho_B> = 0.43; measured 2e-5, 5e-5).
  The collision conserves rho_s, so the kernels give
  the rest population what the eight stored moving populations leave of the
  site's density, and the 16-bit storages round that one population
  stochastically: the only mass error left is the zero-mean rounding of the
  rest population.  Round-to-nearest there drifted by 2.5e-3 (FP16) and 3e-2
  (BF16) in 1000 steps, because the bulk sites of a droplet all round the
  same value the same way.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}      # unit roundoff of the storage
SUBNORMAL = {"f16": 2.0 ** -25, "bf16": 2.0 ** -134}  # half the smallest spacing


def _storage_bound(ref, rho_ref, storage):
    """Elementwise bound of one 16-bit step against the oracle's step of the
    same stored state (see the module docstring)."""
    u, a = UNIT[storage], SUBNORMAL[storage]
    rr = np.asarray(rho_ref, dtype=np.float64)[:, None, None, None]
    dev = np.abs(ref - W9[None, :, None, None] * rr)  # |d*_i| as the storage holds it
    rho = np.abs(ref.sum(axis=1))[:, None]
    bound = u * dev + a + 1e-5 * W9[None, :, None, None] * rho
    moving = (u * dev[:, 1:] + a).sum(axis=1)
    bound[:, 0] = 2 * u * dev[:, 0] + 2 * a + moving + 1e-5 * W9[0] * rho[:, 0]
    return bound


@pytest.mark.parametrize("kernel", ["rows", "tile"])
@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.03)])
@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_one_step_near_reference_state(lb, monkeypatch, kernel, boundary, U, storage):
    st = {"bf16": lb.LB_BF16_DEV, "f16": lb.LB_F16_DEV}[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", kernel)
    nx, ny = 264, 40
    rho_ref = (0.9, 1.1)
    f = inputs.populations(nx, ny, seed=3, base=W9, rel_amp=0.05, species_scale=rho_ref)
    p = lb.make_params(**CFG, boundary=boundary, U_wall=U, storage=st, rho_ref=rho_ref)
    lat = lb.Lattice(nx, ny, p)
    f0 = lat.set_state(f).get_state()  # the stored (rounded) state
    g = lat.step(1).get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, _ = oracle.step(f0, dict(CFG, boundary=boundary, U_wall=U), 1)
    err = np.abs(g - ref)
    bound = _storage_bound(ref, rho_ref, storage)
    worst = float(np.max(err / bound))
    print(f"{kernel} {storage} bd={boundary}: worst error / bound {worst:.2f}", end=" ")
    assert worst <= 1.0
    # the rounding is real: the error exceeds what FP32 arithmetic alone leaves
    assert float(np.max(err / (1e-5 * W9[None, :, None, None] * np.abs(ref.sum(axis=1))[:, None]))) > 1.0


def _walk_bound(storage, steps=1000, sites=512 * 512, rho_mean=0.43):
    ulp = {"f16": 2.0 ** -12, "bf16": 2.0 ** -9}[storage]
    return 4.0 * ulp * np.sqrt(steps / (6.0 * sites)) / rho_mean


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_mass_drift_of_the_droplet_emulsion(lb, storage):
    bound = 1e-6 if storage == "f32" else _walk_bound(storage)
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV}[storage]
    p = lb.make_params(**CFG, storage=st, rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI,
                       init=(0.7, 1.2, 0.1, 0.02))
    lat = lb.Lattice(512, 512, p).init_random(0)
    m0 = lat.observables()["mass"]
    lat.step(1000)
    m1 = lat.observables()["mass"]
    assert lat.status() == lb.LB_OK
    lat.close()
    drift = np.abs(m1[:2] - m0[:2]) / m0[:2]
    assert np.all(drift <= bound), drift
