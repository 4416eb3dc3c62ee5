"""Long-run statistics against the FP64 oracle, and the G = 0 Couette closed form.

A phase-separating emulsion is chaotic: two runs that differ by rounding
diverge site by site within a few hundred steps, so after that only
statistics can be compared.  From the same seeded 128 x 128 droplet emulsion
(Sec. VI couplings) the GPU and the oracle run 2000 steps; the comparison is
on
* the structure factor S(k) of the order parameter rho_A - rho_B, averaged
  over integer shells |k| in [k, k + 1), shells 1..32 (the droplet peak sits
  near k = 11), and its sum over all shells;
* per-species mass drift over the run;
* with Couette walls, the mean shear stress and both wall stresses averaged
  over steps 1000..2000 (every 100 steps).

The G = 0 Couette flow has a closed form (linear u_x between walls moving at
-U and +U, wall stress rho nu 2U/ny); it checks every storage against the
mathematics rather than against the oracle.

Bounds per storage (measured on GB300, then given a margin of ~3x; the
16-bit ones are loose because BF16 keeps 8 and FP16 11 significant bits of
each deviation d_i = f_i - w_i rho_ref, and a weak shear's viscous stress is
a small part of d_i) are in the tables below.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
EMUL = (0.7, 1.2, 0.1, 0.02)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
N, STEPS, SEED, U = 128, 2000, 3, 0.02
WINDOW = range(1000, STEPS + 1, 100)

# storage: (S(k) shells, S total, mass drift, mean stresses)
EMULSION_BOUNDS = {
    "f64": (1e-9, 1e-10, 1e-12, 1e-9),
    "f32": (1e-3, 1e-4, 1e-6, 1e-3),
    "f16": (5e-2, 5e-3, 3e-4, 3e-2),
    "bf16": (0.8, 3e-2, 5e-3, 1.0),
}
# storage: (max |u_x - exact| / U, max |u_y| / U, wall and mean stress relative)
COUETTE_BOUNDS = {
    "f64": (1e-12, 1e-12, 1e-10),
    "f32": (3e-5, 1e-6, 1e-4),
    "f16": (3e-2, 3e-3, 0.1),
    "bf16": (0.2, 3e-3, 0.9),
}


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _storage(lb, name):
    return {"f64": lb.LB_F64, "f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV}[name]


def structure_factor(phi):
    """Shell-averaged |FFT|^2 / sites of phi - <phi>, shells 1 .. n/2 - 1."""
    n = phi.shape[0]
    p = phi - phi.mean()
    F = np.abs(np.fft.fft2(p)) ** 2 / p.size
    k = np.fft.fftfreq(n) * n
    shell = np.floor(np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)).astype(int)
    return np.array([F[shell == s].mean() for s in range(1, n // 2)])


_ORACLE = {}


def _oracle_run(boundary):
    if boundary not in _ORACLE:
        po = dict(CFG, boundary=boundary, U_wall=U if boundary else 0.0)
        f = oracle.init_state(N, N, SEED, oracle.INIT_BERNOULLI, EMUL)
        m0 = oracle.observables(f, po)["mass"]
        t, stress = 0, []
        for t1 in WINDOW:
            f, bad = oracle.step(f, po, t1 - t)
            assert bad == 0
            t = t1
            stress.append(oracle.observables(f, po)["stress"])
        ob = oracle.observables(f, po)
        _ORACLE[boundary] = (m0, ob, np.mean(stress, axis=0))
    return _ORACLE[boundary]


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_emulsion_statistics_match_the_oracle(lb, storage, boundary):
    b_sk, b_tot, b_mass, b_stress = EMULSION_BOUNDS[storage]
    m0_ref, ref, stress_ref = _oracle_run(boundary)
    p = lb.make_params(**CFG, boundary=boundary, U_wall=U if boundary else 0.0,
                       storage=_storage(lb, storage), rho_ref=(0.88, 0.44),
                       init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)
    lat = lb.Lattice(N, N, p).init_random(SEED)
    m0 = lat.observables()["mass"]
    stress = []
    for t1 in WINDOW:
        lat.step(t1 - lat.time)
        stress.append(lat.observables()["stress"])
    ob = lat.observables(fields=True)
    assert lat.status() == lb.LB_OK
    lat.close()
    sk = structure_factor(ob["rho"][0] - ob["rho"][1])
    sk_ref = structure_factor(ref["rho"][0] - ref["rho"][1])
    e_sk = float(np.max(np.abs(sk[:32] / sk_ref[:32] - 1)))
    e_tot = abs(sk.sum() / sk_ref.sum() - 1)
    drift = float(np.max(np.abs(ob["mass"][:2] / m0[:2] - 1)))
    print(f"{storage} bd={boundary}: S(k) {e_sk:.2e} total {e_tot:.2e} drift {drift:.2e}", end=" ")
    assert e_sk <= b_sk
    assert e_tot <= b_tot
    assert drift <= max(b_mass, 4 * float(np.max(np.abs(ref["mass"][:2] / m0_ref[:2] - 1))))
    if boundary:
        e_st = float(np.max(np.abs(np.mean(stress, axis=0) / stress_ref - 1)))
        print(f"stress {e_st:.2e}", end=" ")
        assert e_st <= b_stress


@pytest.mark.parametrize("kernel", ["rows", "tile"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_couette_without_couplings_matches_the_closed_form(lb, monkeypatch, kernel, storage):
    b_ux, b_uy, b_st = COUETTE_BOUNDS[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", kernel)
    nx, ny, Uw = 256, 32, 0.01
    p = lb.make_params(tau=(1.0, 1.0), rho0=0.7, G_AB=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0),
                       boundary=lb.LB_COUETTE, U_wall=Uw, storage=_storage(lb, storage),
                       rho_ref=(1.0, 1.0))
    lat = lb.Lattice(nx, ny, p)
    lat.set_state(np.ones((2, 1, ny, nx)) * W9[None, :, None, None])
    lat.step(20000)  # slowest mode decays as exp(-nu (pi/ny)^2 t): e^-32 of U
    ob = lat.observables(fields=True)
    assert lat.status() == lb.LB_OK
    lat.close()
    exact = Uw * (2 * np.arange(ny) + 1 - ny) / ny
    sigma = 2.0 * (0.5 / 3.0) * 2 * Uw / ny  # total density 2, nu = (tau - 1/2)/3
    e_ux = float(np.max(np.abs(ob["u"][0] - exact[:, None]))) / Uw
    e_uy = float(np.max(np.abs(ob["u"][1]))) / Uw
    e_st = float(np.max(np.abs(ob["stress"] / sigma - 1)))
    print(f"{kernel} {storage}: ux {e_ux:.2e} uy {e_uy:.2e} stress {e_st:.2e}", end=" ")
    assert e_ux <= b_ux
    assert e_uy <= b_uy
    assert e_st <= b_st


# ---- the long cross-checks: 256 x 256, 10^4 steps (emulsion) and
# 5 x 10^3 steps per wall speed (Couette), against the oracle run on the
# host cores ----
#
# FP64 and FP32 stay on the oracle's trajectory over these runs (per-shell
# S(k) differences 3e-13 and 2e-4 measured), so they are held shell by shell.
# The 16-bit runs have decorrelated from it (different droplet arrangements):
# they are held on statistics of the field instead.
# * Bands of shells [1, 8), [8, 16), [16, 32): the periodogram of a random
#   field is exponentially distributed per Fourier mode, so a band of M
#   independent modes (half the lattice modes in it) has a relative standard
#   deviation 1/sqrt(M) from one realisation to the next; two independent
#   realisations differ by sqrt(2)/sqrt(M) (one sd); the bound is four of them.
# * Shells [32, 64) carry the interfaces and the storage's rounding noise:
#   stated bounds (FP16 0.1, BF16 0.3), as for the total S (FP16 5e-3, BF16 3e-2).
# * The droplet peak (shell of the maximum) within 3 shells.
# * Mass drift: the stochastically rounded rest population makes it an
#   unbiased random walk of one rounding (at most one unit in the last place
#   of |d_0| <= 4/9 |rho - rho_ref| ~ 0.36, variance <= ulp^2/6) per site and
#   step: relative sd = ulp sqrt(T / (6 N)) / <rho>; the bound is 4 sd
#   (FP16: ulp 2^-12, BF16: 2^-9, T = 10^4, N = 2^16, <rho> = 0.6).

N2, STEPS2, STEPS_C = 256, 10000, 5000
U_SWEEP = (0.005, 0.02, 0.05)
_ORACLE2 = {}
_ULP = {"f16": 2.0 ** -12, "bf16": 2.0 ** -9}


def _drift_bound(storage, steps):
    if storage == "f64":
        return 1e-11
    if storage == "f32":
        return 2e-6
    return 4.0 * _ULP[storage] * np.sqrt(steps / (6.0 * N2 * N2)) / 0.6


def _band_modes(lo, hi, n=N2):
    k = np.fft.fftfreq(n) * n
    shell = np.floor(np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)).astype(int)
    return int(((shell >= lo) & (shell < hi)).sum()) // 2


def _oracle_long(boundary, U, steps):
    key = (boundary, U, steps)
    if key not in _ORACLE2:
        po = dict(CFG, boundary=boundary, U_wall=U)
        f = oracle.init_state(N2, N2, SEED, oracle.INIT_BERNOULLI, EMUL)
        m0 = oracle.observables(f, po)["mass"]
        t, stress = 0, []
        for t1 in range(steps // 2, steps + 1, steps // 10):
            f, bad = oracle.step(f, po, t1 - t)
            assert bad == 0
            t = t1
            stress.append(oracle.observables(f, po)["stress"])
        _ORACLE2[key] = (m0, oracle.observables(f, po), np.mean(stress, axis=0))
    return _ORACLE2[key]


def _gpu_long(lb, storage, boundary, U, steps):
    p = lb.make_params(**CFG, boundary=boundary, U_wall=U, storage=_storage(lb, storage),
                       rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)
    lat = lb.Lattice(N2, N2, p).init_random(SEED)
    m0 = lat.observables()["mass"]
    stress = []
    for t1 in range(steps // 2, steps + 1, steps // 10):
        lat.step(t1 - lat.time)
        stress.append(lat.observables()["stress"])
    ob = lat.observables(fields=True)
    assert lat.status() == lb.LB_OK
    lat.close()
    return m0, ob, np.mean(stress, axis=0)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_emulsion_256_for_10k_steps_against_the_oracle(lb, storage):
    """The 256^2 x 10^4-step droplet emulsion (the sub-run of the 1024^2 emulsion
    workload): S(k), bands of it, total S, the droplet peak and the mass drift."""
    _, ref, _ = _oracle_long(0, 0.0, STEPS2)
    m0, ob, _ = _gpu_long(lb, storage, 0, 0.0, STEPS2)
    sk = structure_factor(ob["rho"][0] - ob["rho"][1])
    sk_ref = structure_factor(ref["rho"][0] - ref["rho"][1])
    e_sk = float(np.max(np.abs(sk[:64] / sk_ref[:64] - 1)))
    e_tot = abs(sk.sum() / sk_ref.sum() - 1)
    peak, peak_ref = int(np.argmax(sk)), int(np.argmax(sk_ref))
    drift = float(np.max(np.abs(ob["mass"][:2] / m0[:2] - 1)))
    e_band = {}
    for lo, hi in ((1, 8), (8, 16), (16, 32), (32, 64)):
        b = slice(lo - 1, hi - 1)  # sk[j] is shell j + 1
        e_band[(lo, hi)] = abs(sk[b].sum() / sk_ref[b].sum() - 1)
    print(f"{storage}: S(k) {e_sk:.2e} bands {max(e_band.values()):.2e} total {e_tot:.2e} "
          f"peak {peak}/{peak_ref} drift {drift:.2e}", end=" ")
    assert drift <= _drift_bound(storage, STEPS2)
    if storage in ("f64", "f32"):
        b_sk, b_tot = {"f64": (1e-10, 1e-11), "f32": (2e-3, 1e-5)}[storage]
        assert e_sk <= b_sk
        assert e_tot <= b_tot
        assert peak == peak_ref
        return
    for (lo, hi), e in e_band.items():
        if hi <= 32:
            assert e <= 4.0 * np.sqrt(2.0 / _band_modes(lo, hi)), (lo, hi, e)
        else:
            assert e <= {"f16": 0.1, "bf16": 0.3}[storage], (lo, hi, e)
    assert e_tot <= {"f16": 5e-3, "bf16": 3e-2}[storage]
    assert abs(peak - peak_ref) <= 3


# storage: (mean sigma_xy, wall stresses), relative, averaged over the second half
COUETTE_256_BOUNDS = {
    "f64": (1e-10, 1e-10),
    "f32": (1e-4, 5e-3),
    "f16": (3e-3, 0.3),
    "bf16": (3e-2, 0.5),
}


@pytest.mark.parametrize("U", U_SWEEP)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_couette_256_stresses_per_wall_speed_against_the_oracle(lb, storage, U):
    """The droplet emulsion between Couette walls at +-U, U in {0.005, 0.02,
    0.05}, 5000 steps: the FP64 mean shear stress and both wall stresses,
    averaged over the second half of the run, per storage, against the
    oracle's; and the mass drift."""
    _, _, st_ref = _oracle_long(1, U, STEPS_C)
    m0, ob, st = _gpu_long(lb, storage, 1, U, STEPS_C)
    e_st = np.abs(st / st_ref - 1)
    drift = float(np.max(np.abs(ob["mass"][:2] / m0[:2] - 1)))
    print(f"{storage} U={U}: stress {e_st} drift {drift:.2e}", end=" ")
    b_mean, b_wall = COUETTE_256_BOUNDS[storage]
    assert e_st[0] <= b_mean
    assert max(e_st[1], e_st[2]) <= b_wall
    assert st_ref[0] > 0 and min(st_ref[1:]) > 0  # the walls drag the emulsion
    assert drift <= _drift_bound(storage, STEPS_C)
