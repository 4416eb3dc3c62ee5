"""bench.py's multi-rank path, on CPU: two gloo ranks as separate processes.

The path does not shard across GPUs (replicas only), so the only collectives
bench.py makes are barriers and the reductions of the results: the slowest
rank's time, the sum of every rank's site updates, and the gathered request
latencies of the serving workload.  These run here exactly as under torchrun,
with the gloo backend on CPU tensors.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
D = bench.Dist(backend="gloo", device="cpu")
r = D.rank
D.barrier()
seconds = D.max(0.5 + r)                 # rank 1 is the slow one
updates = D.sum(1000 * (r + 1) * 10)     # rank r: (r+1)*1000 sites x 10 steps
lat = D.gather([r, r + 0.5])
out = dict(rank=r, world=D.world, seconds=seconds, updates=updates,
           mlups=bench.whole_job_mlups(updates, seconds), lat=lat)
D.close()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(world, code, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_two_gloo_ranks_reduce_like_the_benchmark():
    outs = _launch(2, WORKER.format(root=ROOT))
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["world"] == 2
        assert d["seconds"] == 1.5  # the slowest rank's time, on every rank
        assert d["updates"] == 30000  # every rank's site updates
        assert d["mlups"] == pytest.approx(30000 / 1.5 / 1e6)
        assert d["lat"] == [0, 0.5, 1, 1.5]  # rank order


def test_reference_arm_runs_on_rank_zero_only():
    # the non-zero ranks of `bench.py --impl reference` under torchrun exit 0
    # without work and print nothing (no process group is formed)
    code = ("import sys; sys.path.insert(0, %r); import bench, types; "
            "bench.run_reference(types.SimpleNamespace(workload='couette4096_f32', steps=1, "
            "warmup=0, cpu_steps=1))" % ROOT)
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_single_rank_needs_no_process_group():
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "D = bench.Dist(backend='gloo', device='cpu'); "
            "print(D.pg is None, D.max(2.5), D.sum(3.0), D.gather([1]))" % ROOT)
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    p = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.split() == ["True", "2.5", "3.0", "[1]"]
