"""Host-side pieces of the serving loop that need no GPU: the Poisson request
generator of the serving workload."""
import numpy as np
import pytest


def test_poisson_requests_recipe():
    try:
        from paper_0906_3611_gb300 import serve, lb
    except ImportError:
        pytest.skip("liblb.so not built")
    sides = list(range(64, 2049, 64))
    reqs = serve.poisson_requests(4000, rate=50.0, seed=0, sides=sides, steps_range=(1e3, 1e5))
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) >= 0)
    assert np.mean(np.diff(arr)) == pytest.approx(1 / 50.0, rel=0.05)
    st = np.array([r.steps for r in reqs])
    assert st.min() >= 1000 and st.max() <= 100000
    assert np.mean(np.log(st)) == pytest.approx(0.5 * (np.log(1e3) + np.log(1e5)), rel=0.02)
    assert set(r.side for r in reqs) <= set(sides)
    frac = np.mean([r.boundary == lb.LB_COUETTE for r in reqs])
    assert frac == pytest.approx(0.5, abs=0.03)
    assert all((r.U_wall == 0.0) == (r.boundary == lb.LB_PERIODIC) for r in reqs)
