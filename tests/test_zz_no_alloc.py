"""lb_observables_noalloc against lb_observables and the FP64 oracle.

lb_observables_noalloc serves callers that cannot call cudaMalloc (their own
pool allocator owns the device memory, or their running stream pipeline must
not take the device-wide synchronisation an allocation can cause).  It keeps
its partial sums in a fixed static device array shared by all calls.  These
tests call it twice in a row, on two different states, for every storage and
both boundaries, and check each result against the handle-based
lb_observables within the tolerances of the other observables tests; FP64
states are also checked against the oracle, and a state with non-positive
densities against the oracle's count of them.  The file is collected last.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
ASYM = dict(tau=(0.8, 1.3), rho0=0.83, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _params(lb, storage, boundary):
    return lb.make_params(**ASYM, boundary=boundary, U_wall=0.04, storage=storage,
                          rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI,
                          init=(0.7, 1.2, 0.1, 0.02))


def _noalloc(lb, lat, p, stream, out):
    cur = lat._bufs[lat.time % 2]  # buffer holding the current state
    lb.lb_observables_noalloc(cur.data_ptr(), lat.nx, lat.ny, (lat.nx + 31) // 32 * 32, p,
                              stream.cuda_stream, out.data_ptr())
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("boundary", [0, 1], ids=["periodic", "couette"])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16dev", "f16dev"])
def test_noalloc_matches_handle_observables_on_two_calls(lb, storage, boundary):
    import torch

    st = {"f64": lb.LB_F64, "f32": lb.LB_F32, "bf16dev": lb.LB_BF16_DEV,
          "f16dev": lb.LB_F16_DEV}[storage]
    nx, ny = 100, 44
    p = _params(lb, st, boundary)
    stream = torch.cuda.Stream()
    lat = lb.Lattice(nx, ny, p, stream=stream)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    lat.init_random(4).step(5)
    for call in range(2):
        ref = lat.observables()
        got = _noalloc(lb, lat, p, stream, out)
        assert np.allclose(got[:2], ref["mass"][:2], rtol=1e-13, atol=0)
        assert np.allclose(got[2:4], ref["mass"][2:], rtol=1e-11, atol=1e-12)
        assert np.allclose(got[4:7], ref["stress"], rtol=1e-10, atol=1e-15)
        assert got[7] == 0.0
        if boundary:
            assert abs(got[5]) > 0.0  # the walls carry stress
        else:
            assert got[5] == 0.0 and got[6] == 0.0
        if st == lb.LB_F64:  # the FP64 state against the oracle's observables
            o = oracle.observables(lat.get_state(), dict(ASYM, boundary=boundary, U_wall=0.04))
            assert np.allclose(got[:2], o["mass"][:2], rtol=1e-13, atol=0)
            assert np.allclose(got[2:4], o["mass"][2:], rtol=1e-11, atol=1e-12)
            assert np.allclose(got[4:7], o["stress"], rtol=1e-10, atol=1e-15)
        lat.step(3)  # a different state for the second call
    lat.close()


def test_noalloc_counts_non_positive_densities_like_the_oracle(lb):
    import torch

    nx, ny = 70, 24
    p = _params(lb, lb.LB_F64, 1)
    f = inputs.populations(nx, ny, seed=9, base=W9, rel_amp=0.05, species_scale=(0.9, 0.5))
    # species A emptied (negative) at three sites, species B at two
    for s, y, x in [(0, 3, 5), (0, 10, 41), (0, 23, 69), (1, 0, 0), (1, 17, 33)]:
        f[s, :, y, x] = -0.01 * W9
    stream = torch.cuda.Stream()
    lat = lb.Lattice(nx, ny, p, stream=stream)
    lat.set_state(f)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        got = _noalloc(lb, lat, p, stream, out)
        o = oracle.observables(f, dict(ASYM, boundary=1, U_wall=0.04))
        assert o["bad"] == 5
        assert got[7] == o["bad"]  # the status word is cleared between calls
        assert np.allclose(got[:2], o["mass"][:2], rtol=1e-13, atol=0)
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_static_area(lb):
    import torch

    p = lb.make_params(storage=lb.LB_F32)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    # 8192 x 4096 needs 131072 tiles of 32 x 8 sites: more than the 65536 it holds
    with pytest.raises(lb.LBError) as e:
        lb.lb_observables_noalloc(f.data_ptr(), 8192, 4096, 8192, p, None, out.data_ptr())
    assert e.value.code == lb.LB_ETOOBIG
