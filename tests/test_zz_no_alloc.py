"""lb_observables_noalloc against lb_observables.

lb_observables_noalloc serves callers that cannot call cudaMalloc (their own
pool allocator owns the device memory, or their running stream pipeline must
not take the device-wide synchronisation an allocation can cause).  It keeps
its partial sums in a fixed static device array shared by all calls.  This
test calls it twice in a row, on two different states, and checks each
result against the handle-based lb_observables within the tolerances of the
other observables tests.  It sits in its own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_noalloc_matches_handle_observables_on_two_calls(lb, storage):
    import torch

    st = {"f64": lb.LB_F64, "f32": lb.LB_F32}[storage]
    nx, ny = 100, 44
    p = lb.make_params(tau=(0.8, 1.3), rho0=0.83, G_AB=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1),
                       boundary=lb.LB_COUETTE, U_wall=0.04, storage=st,
                       init_kind=lb.LB_INIT_BERNOULLI, init=(0.7, 1.2, 0.1, 0.02))
    stream = torch.cuda.Stream()
    lat = lb.Lattice(nx, ny, p, stream=stream)
    pitch = (nx + 31) // 32 * 32
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    lat.init_random(4).step(5)
    for call in range(2):
        ref = lat.observables()
        cur = lat._bufs[lat.time % 2]  # buffer holding the current state
        lb.lb_observables_noalloc(cur.data_ptr(), nx, ny, pitch, p, stream.cuda_stream,
                                  out.data_ptr())
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got[:2], ref["mass"][:2], rtol=1e-13, atol=0)
        assert np.allclose(got[2:4], ref["mass"][2:], rtol=1e-11, atol=1e-12)
        assert np.allclose(got[4:7], ref["stress"], rtol=1e-10, atol=1e-15)
        assert got[7] == 0.0
        assert abs(got[5]) > 0.0  # the walls carry stress
        lat.step(3)  # a different state for the second call
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
