"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

* FP64 storage: one step from identical states agrees to 1e-12 relative, on
  lattices spanning several tiles with ragged tails, the 5 x 5 minimum, both
  boundary kinds, unequal tau and species couplings; 1000 steps of the 64 x 64
  parity configuration are checked step by step from identical states.
* The seeded initial state is bit-identical to the oracle's.
* FP32 storage: max relative density error <= 1e-5 after 100 steps on stable
  states; on the unstable (spinodal) parity configuration every step is
  within 1e-5 of the oracle's and the free run within the envelope of the
  oracle's own propagation of those one-step errors.
* Observables (mass, momentum, sigma_xy, wall stresses, fields) agree to 1e-12.
* At the benchmark size (4096 x 4096 Couette, FP32) sampled sites of one step
  are checked against the oracle run on a local patch (the new populations of
  a site depend only on the 7 x 7 box around it).
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
ASYM = dict(tau=(0.8, 1.3), rho0=0.83, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _params(lb, phys, storage, boundary=0, U=0.0, kind=0, init=(1.0, 1.0, 0.05), rho_ref=(1.0, 1.0)):
    return lb.make_params(tau=phys["tau"], rho0=phys["rho0"], G_AB=phys["G_AB"], Ga=phys["Ga"],
                          Gr=phys["Gr"], boundary=boundary, U_wall=U, storage=storage,
                          rho_ref=rho_ref, init_kind=kind, init=init)


def _oracle_p(phys, boundary=0, U=0.0):
    return dict(phys, boundary=boundary, U_wall=U)


def _rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _scaled_err(g, ref):
    """Error of each population relative to its rest-state scale w_i rho_s(r).

    Late in a phase-separating run populations cross zero (the shifted
    velocity grows where a species is dilute), where an elementwise relative
    error is ill-conditioned: a 2e-16 change of the input already moves such a
    population by ~5e-12 of itself.  Measured against w_i rho_s(r) the same
    input change moves every population by < 2e-14.
    """
    rho = ref.sum(axis=1)
    scale = W9[None, :, None, None] * np.abs(rho[:, None])
    return float(np.max(np.abs(g - ref) / scale))


@pytest.mark.parametrize("kind,init", [(0, (1.0, 1.0, 0.05)), (1, (0.7, 1.2, 0.1, 0.02))])
@pytest.mark.parametrize("shape", [(64, 64), (67, 45)])
def test_seeded_init_is_bit_identical(lb, kind, init, shape):
    nx, ny = shape
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F64, kind=kind, init=init))
    f = lat.init_random(12345).get_state()
    lat.close()
    ref = oracle.init_state(nx, ny, 12345, kind, init)
    assert np.array_equal(f, ref)


# tile kernel: nx below one 128-column strip (or odd); row-streaming kernel: the rest,
# with ragged last strips (264 = 2*128 + 8) and 1..3-row ranges per CTA
SHAPES = [(64, 64), (67, 45), (5, 5), (37, 5), (5, 23), (131, 17),
          (256, 64), (264, 37), (132, 19), (390, 11), (1024, 8)]


@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.03)])
@pytest.mark.parametrize("phys", [CFG, ASYM], ids=["config", "asym"])
@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_one_step_parity(lb, shape, phys, boundary, U):
    nx, ny = shape
    f = inputs.populations(nx, ny, seed=nx * 1000 + ny, base=W9, rel_amp=0.05,
                           species_scale=(0.9, 1.1))
    lat = lb.Lattice(nx, ny, _params(lb, phys, lb.LB_F64, boundary, U))
    lat.set_state(f).step(1)
    g = lat.get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, bad = oracle.step(f, _oracle_p(phys, boundary, U), 1)
    assert bad == 0
    assert _rel_err(g, ref) <= 1e-12


def test_fp64_parity_config_1000_steps_step_by_step(lb):
    """64 x 64, rho = 1 +- 0.05, tau = 1, rho0 = 0.7, G_AB = 0.405, Ga = -9, Gr = 8.1."""
    nx = ny = 64
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F64, init=(1.0, 1.0, 0.05)))
    lat.init_random(0)
    f = oracle.init_state(nx, ny, 0, 0, (1.0, 1.0, 0.05))
    assert np.array_equal(lat.get_state(), f)
    worst = 0.0
    for t in range(1000):
        nxt, bad = oracle.step(f, CFG, 1)
        assert bad == 0
        lat.set_state(f).step(1)
        worst = max(worst, _scaled_err(lat.get_state(), nxt))
        f = nxt
    lat.close()
    assert worst <= 1e-12


def test_fp64_free_run_conserves_mass(lb):
    nx = ny = 64
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F64))
    lat.init_random(1)
    m0 = lat.observables()["mass"]
    lat.step(1000)
    m1 = lat.observables()["mass"]
    assert lat.status() == lb.LB_OK
    lat.close()
    assert np.allclose(m1[:2], m0[:2], rtol=1e-13, atol=0)
    assert np.max(np.abs(m1[2:])) < 1e-10


def _fp32_rho_after(lb, f0, phys, steps, boundary=0, U=0.0, rho_ref=(1.0, 1.0)):
    ny, nx = f0.shape[2:]
    lat = lb.Lattice(nx, ny, _params(lb, phys, lb.LB_F32, boundary, U, rho_ref=rho_ref))
    lat.set_state(f0).step(steps)
    rho = lat.observables(fields=True)["rho"]
    assert lat.status() == lb.LB_OK
    lat.close()
    return rho


def test_fp32_density_error_on_a_stable_state_after_100_steps(lb):
    """FP32 storage and arithmetic: max relative density error <= 1e-5 after 100
    steps, from a relaxed flat interface of the rho0 = 0.7 couplings (a stable
    state, so rounding errors are not amplified).  The deviations are taken
    from the species means (0.61): a reference far from both phases (1.0 for
    the 0.12 phase) costs the dilute phase ~3 bits and gave 2.5e-5."""
    nx, ny = 64, 16
    x = np.arange(nx)
    rA = np.where((x >= 16) & (x < 48), 1.1, 0.12)
    rho = np.stack([np.tile(rA, (ny, 1)), np.tile(1.22 - rA, (ny, 1))])
    f = rho[:, None] * W9[None, :, None, None]
    f, _ = oracle.step(f, CFG, 3000)
    f0 = f.astype(np.float32).astype(np.float64)
    rho_gpu = _fp32_rho_after(lb, f0, CFG, 100, rho_ref=(0.61, 0.61))
    ref = oracle.observables(oracle.step(f0, CFG, 100)[0], CFG)["rho"]
    assert _rel_err(rho_gpu, ref) <= 1e-5


def _storage_scaled_err(g, ref, rho_ref):
    """Error of each population relative to the scale its FP32 deviation is
    stored at, w_i max(rho_s(r), rho_ref,s): the storage holds
    d_i = f_i - w_i rho_ref,s, so a dilute site (rho_s << rho_ref) keeps FP32
    precision relative to w_i rho_ref, not to its own w_i rho_s."""
    rho = np.abs(ref.sum(axis=1))
    rr = np.asarray(rho_ref, dtype=np.float64)[:, None, None]
    scale = W9[None, :, None, None] * np.maximum(rho, rr)[:, None]
    return float(np.max(np.abs(g - ref) / scale))


def _rho_err(f, ref):
    """Max relative density error of state f against state ref."""
    return _rel_err(f.sum(axis=1), ref.sum(axis=1))


def test_fp32_config_run_is_its_one_step_errors_propagated(lb):
    """64 x 64 parity configuration (rho = 1 +- 0.05): the uniform state is
    linearly unstable (spinodal), so any perturbation grows -- in FP64 a single
    1e-7 perturbation of the start reaches ~2e-4 of the density after 100
    steps -- and no FP32 implementation can hold the free run to 1e-5.  The
    bound is derived instead of fixed:

    1. every step of the run, taken by the GPU from the oracle's state (rounded
       to FP32), is within the FP32 bar of the oracle's step: the one-step
       error e_t, measured against the scale each population's deviation is
       stored at, w_i max(rho_s(r), rho_ref,s), is <= 1e-5 (the run separates
       into phases of density 0.03 to 3 around rho_ref = 1);
    2. the oracle propagates those one-step errors: the shadow run
       h_{t+1} = oracle_step(h_t) + e_t injects the GPU's own error fields,
       and seven more runs inject them with random signs per element;
    3. the GPU's free run stays within that ensemble's envelope, max + 4 sd
       over the eight runs, at t = 20, 40, ..., 100 -- a wrong force or
       collision term breaks step 1, and an error growing faster than the
       oracle's own dynamics breaks step 3 at the later times.
    The first 20 steps are also held to 1e-5 directly."""
    nx = ny = 64
    T, marks = 100, (20, 40, 60, 80, 100)
    f0 = oracle.init_state(nx, ny, 0, 0, (1.0, 1.0, 0.05)).astype(np.float32).astype(np.float64)
    traj = [f0]
    for t in range(T):
        traj.append(oracle.step(traj[-1], CFG, 1)[0])
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F32))
    errs = []
    worst = 0.0
    for t in range(T):
        ft = traj[t].astype(np.float32).astype(np.float64)
        g = lat.set_state(ft).step(1).get_state()
        ref = oracle.step(ft, CFG, 1)[0]
        worst = max(worst, _storage_scaled_err(g, ref, (1.0, 1.0)))
        errs.append(g - ref)
    assert lat.status() == lb.LB_OK
    assert worst <= 1e-5  # step 1: the FP32 bar, every step
    # the GPU's free run from the same start
    free = {}
    lat.set_state(f0)
    for t in marks:
        lat.step(t - lat.time)
        free[t] = _rho_err(lat.get_state(), traj[t])
    assert lat.status() == lb.LB_OK
    lat.close()
    assert free[20] <= 1e-5
    # step 2: the oracle's propagation of the one-step errors
    rng = inputs.rng(17)
    members = []
    for k in range(8):
        h = f0.copy()
        d = {}
        for t in range(T):
            e = errs[t] if k == 0 else errs[t] * rng.choice((-1.0, 1.0), size=errs[t].shape)
            h = oracle.step(h, CFG, 1)[0] + e
            if t + 1 in marks:
                d[t + 1] = _rho_err(h, traj[t + 1])
        members.append(d)
    for t in marks:  # step 3
        D = np.array([m[t] for m in members])
        bound = D.max() + 4.0 * D.std()
        assert free[t] <= bound, (t, free[t], D)
    assert free[100] > 1e-5  # (the instability is real: the 1e-5 bar cannot apply here)


def test_fp32_couette_shear_flow_after_100_steps(lb):
    """No couplings, Couette walls: FP32 densities and velocities track FP64."""
    nx, ny = 16, 48
    f0 = inputs.populations(nx, ny, seed=11, base=W9, rel_amp=0.02).astype(np.float32).astype(np.float64)
    phys = dict(tau=(0.9, 0.9), rho0=1.0, G_AB=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0))
    rho_gpu = _fp32_rho_after(lb, f0, phys, 100, boundary=1, U=0.05)
    ref = oracle.observables(oracle.step(f0, _oracle_p(phys, 1, 0.05), 100)[0], _oracle_p(phys, 1, 0.05))
    assert _rel_err(rho_gpu, ref["rho"]) <= 1e-5


@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.04)])
def test_observables_parity_fp64(lb, boundary, U):
    nx, ny = 40, 24
    f = inputs.populations(nx, ny, seed=7, base=W9, rel_amp=0.08, species_scale=(0.8, 1.2))
    p = _oracle_p(ASYM, boundary, U)
    lat = lb.Lattice(nx, ny, _params(lb, ASYM, lb.LB_F64, boundary, U))
    ob = lat.set_state(f).observables(fields=True)
    lat.close()
    ref = oracle.observables(f, p)
    assert np.allclose(ob["mass"][:2], ref["mass"][:2], rtol=1e-13, atol=0)
    assert np.allclose(ob["mass"][2:], ref["mass"][2:], rtol=1e-11, atol=1e-12)
    assert np.allclose(ob["stress"], ref["stress"], rtol=1e-10, atol=1e-15)
    assert _rel_err(ob["rho"], ref["rho"]) <= 1e-13
    assert np.allclose(ob["u"], ref["u"], rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("nx,ny", [(96, 80), (256, 80)])
def test_graph_replay_equals_eager_steps(lb, nx, ny):
    p = _params(lb, CFG, lb.LB_F32, kind=1, init=(0.7, 1.2, 0.1, 0.02))
    a = lb.Lattice(nx, ny, p).init_random(3)
    b = lb.Lattice(nx, ny, p).init_random(3)
    a.step(70)              # graph replays + eager remainder
    for _ in range(70):
        b.step(1)           # eager launches only
    fa, fb = a.get_state(), b.get_state()
    assert a.time == b.time == 70
    a.close()
    b.close()
    assert np.array_equal(fa, fb)


def test_negative_density_is_flagged_like_the_oracle(lb):
    nx, ny = 12, 10
    f = inputs.populations(nx, ny, seed=3, base=W9, rel_amp=0.02, species_scale=(1.0, 1.0))
    f[1, :, 4, 6] = 0.0  # species B empty at one site: no velocity shift there
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F64))
    g = lat.set_state(f).step(1).get_state()
    assert lat.status() == lb.LB_ENEGRHO
    assert lat.status() == lb.LB_OK  # reading clears the word
    lat.close()
    ref, bad = oracle.step(f, CFG, 1)
    assert bad == 1
    assert np.allclose(g, ref, rtol=1e-12, atol=1e-15)


def _patch_rows_cols(ys, xs, ny, nx, boundary, R=5):
    """Rows and columns of the (2R+1)^2 patch around (ys, xs), and the
    boundary the patch is stepped with: the new populations of a site depend
    only on the 7 x 7 box around it, so the centre of an 11 x 11 patch is
    exact (at a Couette wall the patch ends at the wall)."""
    if boundary == 1 and ys < R:
        rows = np.arange(0, 2 * R + 1)
    elif boundary == 1 and ys > ny - 1 - R:
        rows = np.arange(ny - 2 * R - 1, ny)
    else:
        rows = (np.arange(ys - R, ys + R + 1)) % ny
    cols = (np.arange(xs - R, xs + R + 1)) % nx
    pb = boundary if (boundary == 1 and (ys < R or ys > ny - 1 - R)) else 0
    return rows, cols, pb


def _patch_reference(rho0f, ys, xs, ny, nx, phys, boundary, U, dtype, rho_ref=(0.0, 0.0)):
    """One oracle step on a local patch around (ys, xs); returns the centre site's f.
    The initial populations are w_i rho_ref,s + (w_i rho_s - w_i rho_ref,s) rounded
    to `dtype`, as the deviation storages hold them."""
    R = 5
    rows, cols, pb = _patch_rows_cols(ys, xs, ny, nx, boundary, R)
    rho = rho0f[:, rows][:, :, cols]
    base = W9[None, :, None, None] * np.asarray(rho_ref, dtype=np.float64)[:, None, None, None]
    f = base + (W9[None, :, None, None] * rho[:, None] - base).astype(dtype).astype(np.float64)
    g, _ = oracle.step(f, _oracle_p(phys, pb, U), 1)
    cy = int(np.where(rows == ys)[0][0])
    return g[:, :, cy, R]


def test_full_size_sampled_sites_fp32_couette(lb):
    """4096 x 4096 Couette (U = 0.02), FP32, droplet initial state: one step."""
    import torch
    nx = ny = 4096
    U = 0.02
    init = (0.7, 1.2, 0.1, 0.02)
    rho_ref = np.float32([0.87, 0.43]).astype(np.float64)  # the values the library holds
    lat = lb.Lattice(nx, ny, _params(lb, CFG, lb.LB_F32, boundary=1, U=U, kind=1, init=init,
                                     rho_ref=(0.87, 0.43)))
    lat.init_random(0).step(1)
    raw = torch.empty((9, ny, nx, 2), dtype=torch.float32).pin_memory()  # native order [i][y][x][s]
    lb.lb_get_state_raw(lat.h, raw.data_ptr())
    assert lat.status() == lb.LB_OK
    lat.close()
    got = raw.numpy().transpose(3, 0, 1, 2)  # deviations d_i = f_i - w_i rho_ref,s
    base = W9[None, :] * rho_ref[:, None]
    rho0f = oracle.init_densities(nx, ny, 0, 1, init)
    sites = inputs.sample_sites(nx, ny, 40, seed=1) + [(0, 17), (1, 900), (ny - 2, 5), (ny - 1, 2048)]
    for (ys, xs) in sites:
        ref = _patch_reference(rho0f, ys, xs, ny, nx, CFG, 1, U, np.float32, rho_ref)
        assert _rel_err(base + got[:, :, ys, xs].astype(np.float64), ref) <= 1e-5, (ys, xs)


@pytest.mark.parametrize("boundary,U", [(0, 0.0), (1, 0.03)])
@pytest.mark.parametrize("shape", [(520, 41), (136, 9), (4096, 6)])
def test_fp32_one_step_rows_kernel(lb, shape, boundary, U):
    """FP32 storage on the row-streaming kernel: one step within 1e-5 of FP64."""
    nx, ny = shape
    f = inputs.populations(nx, ny, seed=nx + ny, base=W9, rel_amp=0.05, species_scale=(0.9, 1.1))
    f = f.astype(np.float32).astype(np.float64)
    lat = lb.Lattice(nx, ny, _params(lb, ASYM, lb.LB_F32, boundary, U))
    g = lat.set_state(f).step(1).get_state()
    assert lat.status() == lb.LB_OK
    lat.close()
    ref, _ = oracle.step(f, _oracle_p(ASYM, boundary, U), 1)
    assert _rel_err(g, ref) <= 1e-5


def test_tile_and_rows_kernels_agree(lb, monkeypatch):
    """The two step kernels of the library, FP64, 40 steps of a droplet run."""
    nx, ny = 264, 40
    p = _params(lb, CFG, lb.LB_F64, boundary=1, U=0.02, kind=1, init=(0.7, 1.2, 0.1, 0.02))
    out = {}
    for kern in ("tile", "rows"):
        monkeypatch.setenv("LB_STEP_KERNEL", kern)
        lat = lb.Lattice(nx, ny, p).init_random(9).step(40)
        out[kern] = lat.get_state()
        assert lat.status() == lb.LB_OK
        lat.close()
    assert _scaled_err(out["rows"], out["tile"]) <= 1e-11


@pytest.mark.parametrize("n", [15424, 15456])
def test_maximum_size_one_step_fp32(lb, n):
    """The largest square lattice whose nine direction planes the row kernel
    addresses with 32-bit offsets (15424^2: 9 * plane < 2^31 sites), and the
    next size up, which runs on the tile kernel (64-bit offsets).  FP32
    deviation storage, 2 x 17 GB, Couette U = 0.02, asymmetric couplings; the
    state is drawn on the device (U(-1, 1) deviations of 5 % of w_i rho_ref)
    and one step is compared on sampled sites with the oracle on 11 x 11
    patches of that state (1e-5)."""
    import torch
    U = 0.02
    rho_ref = np.float32([0.9, 0.45]).astype(np.float64)
    lat = lb.Lattice(n, n, _params(lb, ASYM, lb.LB_F32, boundary=1, U=U, rho_ref=(0.9, 0.45)))
    pitch = (n + 31) // 32 * 32
    cnt = 9 * n * pitch * 2

    def view(k):
        return lat._bufs[k][:cnt * 4].view(torch.float32).view(9, n, pitch, 2)

    v0 = view(0)
    inputs.fill_device_uniform(v0, seed=n, lo=-1.0, hi=1.0)
    scale = torch.tensor(W9[:, None] * rho_ref[None, :] * 0.05, dtype=torch.float32, device="cuda")
    v0.mul_(scale[:, None, None, :])
    sites = inputs.sample_sites(n, n, 12, seed=3) + [(0, 5), (n - 1, n - 1), (7, 0), (2500, n - 2)]
    patches = []
    for ys, xs in sites:
        rows, cols, pb = _patch_rows_cols(ys, xs, n, n, 1)
        ri = torch.as_tensor(rows, device="cuda")
        ci = torch.as_tensor(cols, device="cuda")
        d = v0.index_select(1, ri).index_select(2, ci).double().cpu().numpy()  # [9][11][11][2]
        patches.append((ys, xs, rows, pb, d.transpose(3, 0, 1, 2)))
    torch.cuda.synchronize()
    lat.step(1).sync()
    assert lat.status() == lb.LB_OK
    v1 = view(1)
    base = W9[None, :] * rho_ref[:, None]
    for ys, xs, rows, pb, d in patches:
        got = base + v1[:, ys, xs, :].double().cpu().numpy().T  # [2][9]
        f = W9[None, :, None, None] * rho_ref[:, None, None, None] + d
        g, bad = oracle.step(f, _oracle_p(ASYM, pb, U), 1)
        assert bad == 0
        ref = g[:, :, int(np.where(rows == ys)[0][0]), 5]
        assert _rel_err(got, ref) <= 1e-5, (ys, xs)
    lat.close()
    del v0, v1, lat
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_mixture_shear_wave_with_unequal_tau(lb, storage, tol):
    """tau_A = 0.6, tau_B = 1.6 (Sec. III footnote: the mixture relaxes with the
    mass-weighted tau_bar): a sine shear wave on the row kernel decays like the
    oracle's, U_k after 100 and 400 steps equal to tol."""
    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    nx, ny, rho = 128, 64, (0.5, 0.5)
    k = 2 * np.pi / ny
    y = np.arange(ny)
    ux = 1e-3 * np.sin(k * y)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cu = cx[None, :, None, None] * ux[None, None, :, None]
    f = (W9[None, :, None, None] * np.asarray(rho)[:, None, None, None] * np.ones((2, 1, ny, nx))
         * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (ux ** 2)[None, None, :, None]))
    if storage == "f32":
        f = f.astype(np.float32).astype(np.float64)
    phys = dict(tau=(0.6, 1.6), rho0=1.0, G_AB=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0))
    lat = lb.Lattice(nx, ny, lb.make_params(**phys, storage=st, rho_ref=rho))
    lat.set_state(f)
    got = []
    for n in (100, 300):
        lat.step(n)
        got.append(lat.shear_diagnostics()["U_k"])
    assert lat.status() == lb.LB_OK
    lat.close()
    g1, _ = oracle.step(f[:, :, :, :4], dict(tau=(0.6, 1.6)), 100)
    g2, _ = oracle.step(g1, dict(tau=(0.6, 1.6)), 300)
    ref = [oracle.shear_diagnostics(g, dict(tau=(0.6, 1.6)))["U_k"] for g in (g1, g2)]
    assert got == pytest.approx(ref, rel=tol)
    nu = np.log(got[0] / got[1]) / (k * k * 300)
    assert nu == pytest.approx((1.1 - 0.5) / 3.0, rel=6e-3)  # tau_bar = 1.1
