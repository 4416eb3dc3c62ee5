"""Continuous-batching server (paper_0906_3611_gb300.serve).

Requests arriving while others run share one resident batch; each served
result must be the same as the request run alone (bitwise, FP32 row kernel),
admission must respect the HBM budget, and the FP64 observables of small
requests must match the oracle.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CFG = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
EMUL = (0.7, 1.2, 0.1, 0.02)


@pytest.fixture(scope="module")
def lbs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_3611_gb300 import lb, serve
    return lb, serve


def _alone(lb, monkeypatch, req):
    monkeypatch.setenv("LB_STEP_KERNEL", "rows")
    p = lb.make_params(**CFG, boundary=req.boundary, U_wall=req.U_wall, storage=lb.LB_F32,
                       rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI, init=EMUL)
    lat = lb.Lattice(req.side, req.side, p).init_random(req.seed).step(req.steps)
    f = lat.get_state()
    lat.close()
    return f


def test_served_results_equal_each_request_alone(lbs, monkeypatch):
    lb, serve = lbs
    R = serve.Request
    reqs = [R(0, 128, 40, 7, lb.LB_PERIODIC, 0.0, 0.00), R(1, 256, 23, 8, lb.LB_COUETTE, 0.03, 0.00),
            R(2, 64, 57, 9, lb.LB_COUETTE, 0.01, 0.02), R(3, 192, 11, 10, lb.LB_PERIODIC, 0.0, 0.03),
            R(4, 128, 33, 11, lb.LB_COUETTE, 0.05, 0.05), R(5, 320, 19, 12, lb.LB_PERIODIC, 0.0, 0.05)]
    srv = serve.Server(CFG, lb.LB_F32, capacity=3, chunk=8, keep_state=True)
    res = srv.run(reqs)
    srv.close()
    assert sorted(r.rid for r in res) == list(range(6))
    for r in res:
        req = reqs[r.rid]
        assert r.steps == req.steps
        assert r.finished >= r.admitted >= r.arrival - 1e-9
        assert np.array_equal(r.state, _alone(lb, monkeypatch, req)), r.rid


def test_admission_respects_the_hbm_budget(lbs):
    lb, serve = lbs
    big = 2 * lb.lb_state_bytes(512, 512, lb.LB_F32)
    reqs = [serve.Request(k, 512, 30 + 5 * k, k, lb.LB_PERIODIC, 0.0, 0.0) for k in range(4)]
    srv = serve.Server(CFG, lb.LB_F32, capacity=4, chunk=16, budget_bytes=1.5 * big)
    with pytest.raises(ValueError):
        srv.submit(serve.Request(99, 1024, 10, 1, lb.LB_PERIODIC, 0.0, 0.0))
    res = sorted(srv.run(reqs), key=lambda r: r.admitted)
    srv.close()
    assert len(res) == 4
    # only one 512^2 request fits at a time: lifetimes do not overlap
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.finished - 1e-6


def test_observables_of_small_requests_match_the_oracle(lbs):
    lb, serve = lbs
    R = serve.Request
    reqs = [R(0, 64, 30, 21, lb.LB_COUETTE, 0.04, 0.0), R(1, 128, 25, 22, lb.LB_PERIODIC, 0.0, 0.0)]
    srv = serve.Server(CFG, lb.LB_F32, capacity=2, chunk=8)
    res = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    for req in reqs:
        f0 = oracle.init_state(req.side, req.side, req.seed, oracle.INIT_BERNOULLI, EMUL)
        f0 = f0.astype(np.float32).astype(np.float64)
        p = dict(CFG, boundary=req.boundary, U_wall=req.U_wall)
        ob = oracle.observables(oracle.step(f0, p, req.steps)[0], p)
        got = res[req.rid]
        assert np.allclose(got.mass[:2], ob["mass"][:2], rtol=1e-6)
        assert np.allclose(got.stress, ob["stress"], rtol=1e-3, atol=1e-7)
