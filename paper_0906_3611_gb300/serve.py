"""Continuous-batching server for lattice Boltzmann simulation requests.

A request asks for `steps` steps of one lattice (side x side, its own seed,
boundary and wall speed).  The server keeps one batched ensemble
(lb_batch_*) resident on the GPU: requests that arrive while others run are
admitted into free slots as long as their population buffers fit the HBM
budget, every chunk of steps advances all admitted requests in one launch
per step, each request stops on the device when its own step budget is
spent, and finished requests are reduced (FP64 mass and stress), returned
and their slots and memory freed before the next chunk.  A request can be
cancelled (queued or running) and can carry a deadline, after which it is
retired unfinished; an admission the device refuses (out of memory, no
free slot) leaves the request queued until memory frees up, or fails it when
nothing else holds memory.

Scheduling only: every step of every request runs in liblb.so's kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import lb


@dataclasses.dataclass
class Request:
    rid: int
    side: int
    steps: int
    seed: int
    boundary: int = lb.LB_PERIODIC
    U_wall: float = 0.0
    arrival: float = 0.0  # seconds after the start of the run
    deadline: float | None = None  # seconds after the start of the run (None: none)


@dataclasses.dataclass
class Result:
    rid: int
    side: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    mass: np.ndarray | None
    stress: np.ndarray | None
    state: np.ndarray | None = None
    status: str = "done"  # done | cancelled | expired | failed

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Admission by HBM budget, one resident batch, chunked stepping.

    The batch's work list starts from `layout` = (layout, longest piece) of
    lb_batch_set_layout, by default contiguous for the 16-bit storages and
    waves of 256-row pieces for FP32; with `retune` the library's autotuner
    picks it again whenever the set of running requests has changed (its
    candidate steps are real steps of every request, so only the slower
    candidates cost time: FP32 serving +10 %, FP16 unchanged)."""

    def __init__(self, phys: dict, storage: int = lb.LB_F32, capacity: int = 64,
                 budget_bytes: float = 150e9, chunk: int = 256, rho_ref=(0.88, 0.44),
                 init_kind: int = lb.LB_INIT_BERNOULLI, init=(0.7, 1.2, 0.1, 0.02),
                 keep_state: bool = False, stream=None, batch=None, layout=None,
                 retune: bool = True):
        self.phys = phys
        self.storage = storage
        self.capacity = capacity
        self.budget = float(budget_bytes)
        self.chunk = int(chunk)
        self.rho_ref = rho_ref
        self.init_kind = init_kind
        self.init = init
        self.keep_state = keep_state
        if batch is None:  # (a caller-supplied batch object stands in for the device one)
            import torch
            self.stream = stream if stream is not None else torch.cuda.Stream()
            batch = lb.Batch(capacity, storage, self.stream)
        self.batch = batch
        if layout is None:  # measured on 48 Poisson requests of 64..2048 sites a side
            layout = (0, 1 << 30) if storage in (lb.LB_BF16_DEV, lb.LB_F16_DEV) else (2, 256)
        if hasattr(self.batch, "set_layout"):
            self.batch.set_layout(*layout)
        self.retune = retune and hasattr(self.batch, "autotune")
        self._tuned_for = None  # the running (slot, request) set the work list was tuned for
        self.queue: collections.deque[Request] = collections.deque()
        self.active: dict[int, tuple[Request, float]] = {}  # slot -> (request, admitted)
        self.used = 0.0
        self.site_updates = 0
        self.admission_failures = 0
        self.retired: list[Result] = []  # cancelled / expired / failed, not yet returned
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def bytes_of(self, req: Request) -> int:
        return 2 * lb.lb_state_bytes(req.side, req.side, self.storage)

    def params(self, req: Request) -> lb.lb_params:
        return lb.make_params(**self.phys, boundary=req.boundary, U_wall=req.U_wall,
                              storage=self.storage, rho_ref=self.rho_ref,
                              init_kind=self.init_kind, init=self.init)

    def submit(self, req: Request):
        if self.bytes_of(req) > self.budget:
            raise ValueError(f"request {req.rid} needs more than the whole HBM budget")
        self.queue.append(req)

    def _retire(self, req: Request, admitted: float, status: str, steps: int = 0):
        self.retired.append(Result(req.rid, req.side, steps, req.arrival, admitted, self.now(),
                                   None, None, None, status))

    def admit(self) -> int:
        """Move queued requests into free slots while their memory fits (FIFO).
        A refused admission (LB_ENOMEM, LB_EBUSY) keeps the request at the head
        of the queue while other requests hold memory, and fails it otherwise."""
        n = 0
        while self.queue and len(self.active) < self.capacity:
            req = self.queue[0]
            need = self.bytes_of(req)
            if self.used + need > self.budget:
                break
            try:
                slot = self.batch.add(req.side, req.side, self.params(req), req.seed, req.steps)
            except lb.LBError as e:
                if e.code not in (lb.LB_ENOMEM, lb.LB_EBUSY):
                    raise
                self.admission_failures += 1
                if not self.active:  # nothing to wait for: it can never be admitted
                    self.queue.popleft()
                    self._retire(req, self.now(), "failed")
                    continue
                break
            self.queue.popleft()
            self.active[slot] = (req, self.now())
            self.used += need
            n += 1
        return n

    def cancel(self, rid: int) -> bool:
        """Withdraw request `rid`, queued or running; False if it is unknown or done."""
        for req in list(self.queue):
            if req.rid == rid:
                self.queue.remove(req)
                self._retire(req, self.now(), "cancelled")
                return True
        for slot, (req, admitted) in list(self.active.items()):
            if req.rid == rid:
                self._release(slot, req)
                self._retire(req, admitted, "cancelled")
                return True
        return False

    def _release(self, slot: int, req: Request):
        self.batch.remove(slot)
        del self.active[slot]
        self.used -= self.bytes_of(req)

    def expire(self) -> int:
        """Retire every queued or running request whose deadline has passed."""
        t, n = self.now(), 0
        for req in [r for r in self.queue if r.deadline is not None and r.deadline <= t]:
            self.queue.remove(req)
            self._retire(req, t, "expired")
            n += 1
        for slot, (req, admitted) in list(self.active.items()):
            if req.deadline is not None and req.deadline <= t:
                self._release(slot, req)
                self._retire(req, admitted, "expired")
                n += 1
        return n

    def step_chunk(self) -> list[Result]:
        """Advance every admitted request by up to `chunk` steps; retire the finished."""
        if not self.active:
            return []
        running = frozenset((slot, req.rid) for slot, (req, _) in self.active.items())
        if self.retune and running != self._tuned_for:
            self.batch.autotune(2)
            self._tuned_for = running
        self.batch.run(self.chunk)
        remaining, done = self.batch.poll()
        status = self.batch.status()
        if status not in (lb.LB_OK, lb.LB_ENEGRHO):
            raise lb.LBError(status, "batch step")
        out = []
        for slot, (req, admitted) in list(self.active.items()):
            if remaining[slot] > 0:
                continue
            obs = self.batch.observables(slot)
            state = self.batch.get_state(slot) if self.keep_state else None
            out.append(Result(req.rid, req.side, int(done[slot]), req.arrival, admitted, self.now(),
                              obs["mass"], obs["stress"], state))
            self._release(slot, req)
            self.site_updates += req.side * req.side * req.steps
        return out

    def run(self, requests: list[Request], time_limit: float | None = None) -> list[Result]:
        """Serve requests arriving at their `arrival` times (seconds from now)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = time.perf_counter()
        results: list[Result] = []
        while pending or self.queue or self.active:
            t = self.now()
            if time_limit is not None and t > time_limit:
                break
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            self.expire()
            self.admit()
            results.extend(self.retired)
            self.retired = []
            if self.active:
                results.extend(self.step_chunk())
            elif pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - self.now())))
        results.extend(self.retired)
        self.retired = []
        return results

    def close(self):
        self.batch.close()


def poisson_requests(n: int, rate: float, seed: int, sides, steps_range, couette_fraction=0.5,
                     umax: float = 0.05) -> list[Request]:
    """n requests with exponential inter-arrival times (mean 1/rate), sides drawn
    uniformly from `sides`, steps log-uniform in steps_range, periodic or Couette
    with probability couette_fraction, U uniform in [0, umax]."""
    g = np.random.Generator(np.random.Philox(key=seed))
    arrivals = np.cumsum(g.exponential(1.0 / rate, size=n))
    side = g.choice(np.asarray(sides), size=n)
    lo, hi = np.log(steps_range[0]), np.log(steps_range[1])
    steps = np.exp(g.uniform(lo, hi, size=n)).astype(np.int64)
    couette = g.uniform(size=n) < couette_fraction
    U = g.uniform(0.0, umax, size=n)
    return [Request(rid=k, side=int(side[k]), steps=int(steps[k]), seed=1000 + k,
                    boundary=lb.LB_COUETTE if couette[k] else lb.LB_PERIODIC,
                    U_wall=float(U[k]) if couette[k] else 0.0, arrival=float(arrivals[k]))
            for k in range(n)]
