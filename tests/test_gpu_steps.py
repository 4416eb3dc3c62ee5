"""The ways a lattice is stepped agree bit for bit.

A lattice stepped n times in one call replays captured graphs of 32 steps
and launches the rest one by one; stepped one step per call, it launches
every step alone; run as a batch replica, it goes through the batched
kernel, which splits the rows into other work items.  The per-site
arithmetic does not depend on any of this, so all three must agree bit for
bit, across graph boundaries, odd step counts and the buffer parity they
leave, in every storage and for both boundaries.  The row kernel's two CTA
shapes (FP32 and the 16-bit storages) cut the lattice into different strips
and ranges and give the same bits too; the shape autotuner leaves the state, the step count and the
status word as they were.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
EMUL = (0.7, 1.2, 0.1, 0.02)


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb as _lb
    return _lb


def _p(lb, storage, boundary):
    return lb.make_params(**CFG, boundary=boundary, U_wall=0.03 if boundary else 0.0,
                          storage=storage, rho_ref=(0.88, 0.44),
                          init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)


@pytest.mark.parametrize("boundary", [0, 1], ids=["periodic", "couette"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f64"])
def test_one_call_equals_single_steps_and_the_batched_kernel(lb, monkeypatch, storage, boundary):
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV, "f64": lb.LB_F64}[storage]
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    nx, ny, seed, n = 384, 72, 21, 131  # 131 = 4 x 32 + 3: four graph replays, odd parity
    p = _p(lb, st, boundary)
    a = lb.Lattice(nx, ny, p).init_random(seed).step(n)
    fa = a.get_state()
    assert a.status() == lb.LB_OK
    b = lb.Lattice(nx, ny, p).init_random(seed)
    for _ in range(n):
        b.step(1)
    fb = b.get_state()
    assert b.status() == lb.LB_OK
    a.close()
    b.close()
    assert np.array_equal(fa, fb)
    bt = lb.Batch(2, st)
    slot = bt.add(nx, ny, p, seed, n)
    bt.run(n)
    fc = bt.get_state(slot)
    assert bt.status() == lb.LB_OK
    bt.close()
    assert np.array_equal(fa, fc)


@pytest.mark.parametrize("boundary", [0, 1], ids=["periodic", "couette"])
@pytest.mark.parametrize("nx", [500, 1024])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_the_wide_cta_shape_gives_the_same_bits(lb, monkeypatch, storage, nx, boundary):
    # shape 1 (FP32: 224-column strips of 7 compute warps; 16-bit: 256-column
    # strips of 8) against shape 0 (128-column strips of 4); nx = 500 leaves a
    # ragged last strip in both
    st = {"f32": lb.LB_F32, "f16": lb.LB_F16_DEV, "bf16": lb.LB_BF16_DEV}[storage]
    p = _p(lb, st, boundary)
    ny, n = 96, 45
    out = []
    for shape in ("0", "1"):
        monkeypatch.setenv("LB_ROW_SHAPE", shape)
        lat = lb.Lattice(nx, ny, p)
        assert lat.row_shape == int(shape)
        out.append(lat.init_random(8).step(n).get_state())
        assert lat.status() == lb.LB_OK
        lat.close()
    assert np.array_equal(out[0], out[1])


def test_autotune_keeps_the_state_and_reports_the_shape(lb, monkeypatch):
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    p = _p(lb, lb.LB_F32, 1)
    a = lb.Lattice(640, 200, p).init_random(4).step(9)
    f = a.get_state()
    shape = a.autotune(3)
    assert shape in (0, 1) and a.row_shape == shape
    assert np.array_equal(a.get_state(), f)
    assert a.time == 9 and a.status() == lb.LB_OK
    g = a.step(30).get_state()
    b = lb.Lattice(640, 200, p).init_random(4).step(39)
    assert np.array_equal(b.get_state(), g)
    a.close()
    b.close()


def test_shape_forcing_and_the_tile_kernel(lb, monkeypatch):
    monkeypatch.setenv("LB_ROW_SHAPE", "1")
    with pytest.raises(lb.LBError) as e:  # no wide shape for FP64
        lb.Lattice(512, 64, _p(lb, lb.LB_F64, 0))
    assert e.value.code == lb.LB_EINVAL
    monkeypatch.delenv("LB_ROW_SHAPE")
    monkeypatch.setenv("LB_STEP_KERNEL", "tile")
    lat = lb.Lattice(512, 64, _p(lb, lb.LB_F32, 0))
    assert lat.row_shape == -1
    assert lat.autotune(2) == -1
    lat.close()


def test_autotune_refuses_while_the_stream_is_captured(lb, monkeypatch):
    import torch

    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    lat = lb.Lattice(640, 200, _p(lb, lb.LB_F32, 1)).init_random(2)
    lat.sync()
    shape = lat.row_shape
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=lat.stream):
        x = torch.zeros(4, device="cuda")
        x += 1.0
        with pytest.raises(lb.LBError) as e:
            lat.autotune(2)
    assert e.value.code == lb.LB_EBUSY
    g.replay()
    torch.cuda.synchronize()
    assert lat.row_shape == shape and lat.status() == lb.LB_OK
    lat.close()
