"""Host-side pieces of the serving loop that need no GPU: the Poisson request
generator of the serving workload, and the scheduler (admission by budget and
slots, cancellation, deadlines, refused admissions and device errors) on a
stand-in batch, with the failures injected on the host."""
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


# ---- the scheduler on a stand-in batch (no GPU): admission, cancellation,
# deadlines and refused admissions (injected on the host) ----

class FakeBatch:
    """Stands in for lb.Batch: run(n) spends up to n steps of every replica's
    budget; `fail_adds` admissions raise LBError(code) first (injected)."""

    def __init__(self, lb, capacity, fail_adds=0, code=None):
        self.lb, self.capacity = lb, capacity
        self.slots = {}
        self.fail_adds = fail_adds
        self.code = lb.LB_ENOMEM if code is None else code
        self.status_code = lb.LB_OK

    def add(self, nx, ny, params, seed, steps):
        if self.fail_adds > 0:
            self.fail_adds -= 1
            raise self.lb.LBError(self.code, "lb_batch_add")
        k = min(set(range(self.capacity)) - set(self.slots))
        self.slots[k] = [int(steps), 0]
        return k

    def remove(self, k):
        del self.slots[k]

    def run(self, n):
        for v in self.slots.values():
            d = min(n, v[0])
            v[0] -= d
            v[1] += d

    def poll(self):
        rem = np.full(self.capacity, -1, dtype=np.int64)
        done = np.full(self.capacity, -1, dtype=np.int64)
        for k, (r, d) in self.slots.items():
            rem[k], done[k] = r, d
        return rem, done

    def status(self):
        return self.status_code

    def observables(self, k):
        return {"mass": np.ones(4), "stress": np.zeros(3)}

    def get_state(self, k):
        return None

    def close(self):
        pass


@pytest.fixture()
def srvmod():
    try:
        from paper_0906_3611_gb300 import lb, serve
    except ImportError:
        pytest.skip("liblb.so not built")
    return lb, serve


PHYS = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))


def _server(lb, serve, capacity=4, budget_sides=None, fail_adds=0, code=None, chunk=10):
    fb = FakeBatch(lb, capacity, fail_adds, code)
    budget = 1e15 if budget_sides is None else sum(
        2 * lb.lb_state_bytes(s, s, lb.LB_F32) for s in budget_sides)
    return serve.Server(PHYS, lb.LB_F32, capacity=capacity, chunk=chunk, budget_bytes=budget,
                        batch=fb), fb


def test_admission_by_budget_and_capacity(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=3, budget_sides=(256, 256))
    for k in range(4):
        srv.submit(serve.Request(k, 256, 25 + 10 * k, k))
    assert srv.admit() == 2 and len(srv.queue) == 2  # the budget holds two
    out = srv.step_chunk() + srv.step_chunk() + srv.step_chunk()
    assert [r.rid for r in out] == [0] and srv.used > 0  # request 0 (25 steps) is done
    assert srv.admit() == 1 and [req.rid for req, _ in srv.active.values()] == [1, 2]
    with pytest.raises(ValueError):  # larger than the whole budget
        srv.submit(serve.Request(9, 1024, 5, 9))


def test_cancel_queued_and_running_requests(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=1)
    srv.submit(serve.Request(0, 128, 100, 0))
    srv.submit(serve.Request(1, 128, 100, 1))
    srv.admit()
    assert srv.cancel(1) and srv.cancel(0) and not srv.cancel(7)
    assert not srv.active and not srv.queue and srv.used == 0 and not fb.slots
    assert sorted((r.rid, r.status) for r in srv.retired) == [(0, "cancelled"), (1, "cancelled")]


def test_deadlines_expire_queued_and_running_requests(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=1, chunk=5)
    reqs = [serve.Request(0, 128, 10**9, 0, deadline=0.05),  # runs, then expires
            serve.Request(1, 128, 10, 1, deadline=0.0),      # expires in the queue
            serve.Request(2, 128, 10, 2)]
    res = srv.run(reqs, time_limit=30.0)
    st = {r.rid: r.status for r in res}
    assert st == {0: "expired", 1: "expired", 2: "done"}
    assert next(r for r in res if r.rid == 2).steps == 10
    assert not fb.slots and srv.used == 0


def test_refused_admission_waits_while_memory_is_held(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=2, chunk=10)
    srv.submit(serve.Request(0, 128, 20, 0))
    srv.admit()
    fb.fail_adds = 1  # the device refuses the next admission once
    srv.submit(serve.Request(1, 128, 20, 1))
    assert srv.admit() == 0 and srv.admission_failures == 1 and len(srv.queue) == 1
    assert srv.admit() == 1  # memory freed up: admitted on the retry
    res = srv.run([], time_limit=30.0)
    assert sorted(r.rid for r in res if r.status == "done") == [0, 1]


def test_refused_admission_with_nothing_running_fails_the_request(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=2, fail_adds=1, code=None)
    res = srv.run([serve.Request(0, 128, 20, 0), serve.Request(1, 128, 20, 1, arrival=0.01)],
                  time_limit=30.0)
    assert {r.rid: r.status for r in res} == {0: "failed", 1: "done"}


def test_other_device_errors_propagate(srvmod):
    lb, serve = srvmod
    srv, fb = _server(lb, serve, capacity=2, fail_adds=1, code=lb.LB_ECUDA)
    srv.submit(serve.Request(0, 128, 20, 0))
    with pytest.raises(lb.LBError):
        srv.admit()
    srv2, fb2 = _server(lb, serve, capacity=2)
    srv2.submit(serve.Request(0, 128, 20, 0))
    srv2.admit()
    fb2.status_code = lb.LB_ETIMEOUT  # a bounded device wait gave up
    with pytest.raises(lb.LBError):
        srv2.step_chunk()
