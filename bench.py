"""Throughput benchmark of the fused two-species lattice Boltzmann step.

Default workload (one GPU): 4096 x 4096 Couette lattice, walls at +-U with
U = 0.02, FP32 populations, seeded Bernoulli(0.7) droplet mixture, the
rho0 = 0.7 couplings (G_AB = 0.405, G^a = -9, G^r = 8.1), tau = 1.  A step is
one lb_step of the whole lattice (all 2 x 2^24 site updates); the metric is
MLUPS (million two-species site updates per second).  Each population buffer
is 1.21 GB, far larger than the 129 MB L2, so no flush is needed between steps.

Multi-GPU (torchrun): independent replicas, one lattice per rank (weak
scaling, no data-path collective); value = all ranks' site updates / the
slowest rank's time.

--impl reference times the FP64 CPU oracle instead (the baseline arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PHYS = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-9.0, -9.0), Gr=(8.1, 8.1))
INIT = (0.7, 1.2, 0.1, 0.02)
WORKLOADS = {
    # name: (nx, ny, boundary, U, storage)
    "couette4096_f32": (4096, 4096, 1, 0.02, 1),
    "emulsion1024_f32": (1024, 1024, 0, 0.0, 1),
    "couette2048_f32": (2048, 2048, 1, 0.02, 1),
    "couette4096_bf16dev": (4096, 4096, 1, 0.02, 2),
    "couette4096_f16dev": (4096, 4096, 1, 0.02, 3),
    "couette2048_bf16dev": (2048, 2048, 1, 0.02, 2),
    "couette2048_f16dev": (2048, 2048, 1, 0.02, 3),
}
BATCHES = {
    # name: (replicas, side choices, U range, storage)
    "batch256_f32": (256, (128, 256, 512, 1024), 0.05, 1),
    "batch256_f16dev": (256, (128, 256, 512, 1024), 0.05, 3),
    # the same size mix at a quarter of the replicas (1.6 GB: the profiling case)
    "batch64_f16dev": (64, (128, 256, 512, 1024), 0.05, 3),
    "batch64_f32": (64, (128, 256, 512, 1024), 0.05, 1),
}
SHEARS = {
    # name: (replicas, side, U0 (laminar amplitude of the Kolmogorov flow), storage)
    # the paper's shear ensemble (Sec. VII-VIII): 128^2 lattices, rho0 = 0.7 standard
    # couplings, <rho> = 0.612 +- 0.01, body force g = U0 nu k^2 at k = 2 pi / 128
    "shear100x128_f32": (100, 128, 0.03, 1),
}
STD07 = dict(tau=(1.0, 1.0), rho0=0.7, G_AB=0.405, Ga=(-15.0, -14.0), Gr=(14.1, 13.1))
SERVES = {
    # name: (storage, requests, rate per s, sides, steps range, HBM budget, slots, chunk)
    "serve_f32": (1, 48, 50.0, tuple(range(64, 2049, 64)), (1e3, 1e5), 150e9, 64, 256),
    "serve_f16dev": (3, 48, 50.0, tuple(range(64, 2049, 64)), (1e3, 1e5), 150e9, 64, 256),
}
MIXES = {
    # name: (nx, ny, storage): three species on a periodic lattice -- the A/B
    # emulsion couplings (rho0 = 0.7, G^a = -9, G^r = 8.1, G_AB = 0.405) and a
    # dilute third species C without self couplings, coupled to both by
    # G_AC = G_BC = 0.2; rho = (1, 1, 0.1) +- (0.05, 0.05, 0.01)
    "mix3_4096_f32": (4096, 4096, 1),
    "mix3_1024_f32": (1024, 1024, 1),
}
MIX3 = dict(ns=3, tau=[1.0, 1.0, 1.0], rho0=0.7, Ga=[-9.0, -9.0, 0.0], Gr=[8.1, 8.1, 0.0],
            G=[[0.0, 0.405, 0.2], [0.405, 0.0, 0.2], [0.2, 0.2, 0.0]])
MIX3_INIT = ([1.0, 1.0, 0.1], [0.05, 0.05, 0.01])
STORAGE_NAME = {0: "f64", 1: "f32", 2: "bf16dev", 3: "f16dev"}
ELEM = {0: 8, 1: 4, 2: 2, 3: 2}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while work runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClocks:
    """In-process NVML samples of the SM clock, power and clock-event reasons,
    taken every ~10 ms on a background thread (libnvidia-ml through ctypes;
    reads only).  Samples taken while `loaded` is set (the timed region) are the
    under-load samples.  Falls back to the nvidia-smi sampler without NVML."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, local: int, period_s: float = 0.01):
        import ctypes
        import threading
        self.period = period_s
        self.samples = []  # (loaded, sm_mhz, power_w, reasons bitmask)
        self.loaded = False
        self.fallback = None
        self._stop = threading.Event()
        self._thread = None
        self.lib = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            ok = False
            try:
                import torch
                pr = torch.cuda.get_device_properties(local)
                bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
            except Exception:
                ok = False
            if not ok:
                vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
                idx = int(vis.split(",")[local]) if vis and vis.split(",")[0].isdigit() else local
                if lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(h)) != 0:
                    raise OSError("nvmlDeviceGetHandle")
            self.h = h
            self.lib = lib
            self.ct = ctypes
            self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        except Exception:
            self.lib = None
            self.fallback = ClockSampler(local)

    def _sample(self):
        ct = self.ct
        mhz, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz))
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
        self.reason_fn(self.h, ct.byref(rs))
        self.samples.append((self.loaded, float(mhz.value), mw.value / 1e3, int(rs.value)))

    def _run(self):
        while not self._stop.is_set():
            try:
                self._sample()
            except Exception:
                pass
            time.sleep(self.period)

    def start(self):
        if self.fallback is not None:
            self.fallback.start()
            return
        import threading
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    def stop(self) -> dict:
        if self.fallback is not None:
            return self.fallback.stop()
        self._stop.set()
        self._thread.join(timeout=2)
        load = [x for x in self.samples if x[0]]
        use = load or self.samples
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"],
                    "samples": 0, "samples_under_load": 0, "source": "nvml"}
        reasons = set()
        for x in use:
            for bit, nm in self.REASONS.items():
                if x[3] & bit:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(x[1] for x in use), "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(x[1] for x in use), "power_w_max": max(x[2] for x in use),
                "reasons": sorted(reasons), "samples": len(self.samples),
                "samples_under_load": len(load), "source": "nvml, 10 ms"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """One process per GPU under torchrun.  The path does not shard: every rank
    runs its own replica(s), and the only collectives are the barriers around
    the timed region and the reductions of the results below (NCCL on GPUs;
    gloo with device "cpu" in the CPU tests)."""

    def __init__(self, backend: str = "nccl", device: str = "cuda"):
        self.rank, self.world, self.local = dist_env()
        self.device = device
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()
        if self.pg is not None:
            self.pg.barrier()
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()

    def _reduce(self, x: float, op: str) -> float:
        if self.pg is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=getattr(self.pg.ReduceOp, op))
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, "MAX")

    def sum(self, x: float) -> float:
        return self._reduce(x, "SUM")

    def gather(self, xs: list) -> list:
        """Concatenation of every rank's list (rank order)."""
        if self.pg is None:
            return list(xs)
        out = [None] * self.world
        self.pg.all_gather_object(out, list(xs))
        return [v for part in out for v in part]

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()
            self.pg = None


def whole_job_mlups(site_updates_all_ranks: float, seconds_slowest_rank: float) -> float:
    """Whole-job throughput: every rank's site updates over the slowest rank's time."""
    return site_updates_all_ranks / seconds_slowest_rank / 1e6


def cpu_baseline_run(nx, ny, boundary, U, steps):
    """Time the FP64 oracle (as it stands) on the host cores."""
    import oracle
    p = dict(PHYS, boundary=boundary, U_wall=U)
    f = oracle.init_state(nx, ny, 0, oracle.INIT_BERNOULLI, INIT)
    t0 = time.perf_counter()
    oracle.step(f, p, steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt, oracle.max_threads()


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    nx, ny, boundary, U, storage = WORKLOADS[args.workload]
    # each step: one oracle step of a 1024 x 1024 sample of the workload (same physics,
    # boundary and initial recipe); bounded so the whole run takes a few minutes
    sx = sy = 1024
    import oracle
    p = dict(PHYS, boundary=boundary, U_wall=U)
    f = oracle.init_state(sx, sy, 0, oracle.INIT_BERNOULLI, INIT)
    f, _ = oracle.step(f, p, args.warmup)
    t0 = time.perf_counter()
    f, _ = oracle.step(f, p, args.steps)
    dt = time.perf_counter() - t0
    mlups = sx * sy * args.steps / dt / 1e6
    cores = oracle.max_threads()
    sample = f"FP64 oracle, {sx}x{sy} sample of {args.workload} per step, OpenMP {cores} threads"
    line = {"impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nx": nx, "ny": ny, "sample_nx": sx,
                       "sample_ny": sy},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def timed_blocks(D, stream, fn, reps, clocks=None, target_s=None):
    """Time blocks of work: each block is fn() (K steps enqueued on `stream`),
    bracketed by a barrier and a device synchronize, timed with CUDA events on
    that stream; a block's time is the max over ranks.  With `target_s` the
    repetition count grows from `reps` until about that many seconds are
    timed.  Returns the list of block times (ms)."""
    import torch

    out = []
    r = 0
    while True:
        D.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        if clocks is not None:
            clocks.loaded = True
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        if clocks is not None:
            clocks.loaded = False
        D.barrier()
        out.append(D.max(a.elapsed_time(b)))
        r += 1
        if r == 1 and target_s:  # size the run from the first block
            reps = int(D.max(max(reps, min(4000, int(target_s * 1e3 / max(out[0], 1e-3))))))
        if r >= reps:
            return out


def lattice_params(lb, storage, boundary, U):
    return lb.make_params(**PHYS, boundary=boundary, U_wall=U, storage=storage,
                          rho_ref=(0.87, 0.43), init_kind=lb.LB_INIT_BERNOULLI, init=INIT)


def single_lattice(lb, D, name, steps, warmup, seed, reps=25, target_s=1.5, clocks=None, U=None):
    """MLUPS of one lattice workload: the median over repeated blocks of `steps`
    graph-replayed steps.  Returns (dict, lattice, stream)."""
    import torch

    nx, ny, boundary, U0, storage = WORKLOADS[name]
    U = U0 if U is None else U
    stream = torch.cuda.Stream()
    lat = lb.Lattice(nx, ny, lattice_params(lb, storage, boundary, U), stream=stream)
    lat.init_random(seed)
    lat.step(warmup)
    lat.sync()
    ms = timed_blocks(D, stream, lambda: lat.step(steps), reps, clocks, target_s)
    med = statistics.median(ms)
    bps = 2 * 18 * ELEM[storage]  # 18 populations read + 18 written per site
    peak, peak_kind = peaks()
    achieved = bps * nx * ny / (med * 1e-3 / steps) / 1e9
    out = {"workload": name, "mlups": whole_job_mlups(D.sum(nx * ny * steps), med * 1e-3),
           "ms_per_step": med / steps, "blocks": len(ms), "steps_per_block": steps,
           "ms_block_min_max": [min(ms), max(ms)], "bytes_per_site": bps,
           "achieved_gbs": achieved, "frac": achieved / peak, "peak_gbs": peak,
           "peak_kind": peak_kind, "status": lb.lb_strerror(lat.status()),
           "row_shape": lat.row_shape}
    return out, lat, stream


def run_gpu(args):
    import numpy as np
    import torch

    from paper_0906_3611_gb300 import lb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    nx, ny, boundary, U, storage = WORKLOADS[args.workload]
    sites = nx * ny
    clocks = NvmlClocks(local)
    clocks.start()
    res, lat, stream = single_lattice(lb, D, args.workload, args.steps, args.warmup, rank,
                                      reps=args.reps, target_s=args.target_s, clocks=clocks)
    clocks_d = clocks.stop()
    ms = res["ms_per_step"] * args.steps  # median block time, max over ranks
    value = res["mlups"]

    # end-to-end through the C ABI with host buffers: pinned host state -> device,
    # K steps, FP64 observables back to the host
    es = ELEM[storage]
    host = torch.empty(2 * 9 * ny * nx * es, dtype=torch.uint8).pin_memory()
    lb.lb_get_state_raw(lat.h, host.data_ptr())
    mass = np.zeros(4)
    stress = np.zeros(3)
    e2e = []
    for _ in range(3):
        D.barrier()
        t0 = time.perf_counter()
        lb.lb_set_state_raw(lat.h, host.data_ptr())
        lb.lb_step(lat.h, args.steps)
        lb.lb_observables(lat.h, None, None, stress, mass)
        e2e.append(D.max(time.perf_counter() - t0))
    e2e_value = whole_job_mlups(D.sum(sites * args.steps), statistics.median(e2e))
    status = lat.status()
    lat.close()

    bytes_per_site = res["bytes_per_site"]
    achieved = res["achieved_gbs"]
    peak, peak_kind = res["peak_gbs"], res["peak_kind"]
    traffic = None
    tr = {}
    prof = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(prof):
        from paper_0906_3611_gb300 import build as _b
        sha = _b.rows_kernel_sha()
        for line in open(prof):
            if line.startswith(f"{args.workload} ") and "kernel_sha=" in line:
                parts = dict(kv.split("=", 1) for kv in line.split()[1:] if "=" in kv)
                if parts.get("kernel_sha") == sha:
                    tr = parts
                    traffic = float(parts["read_bytes"]) + float(parts["write_bytes"])

    extra = None
    if world == 1 and not args.no_extra and args.workload == "couette4096_f32":
        # the reduced-storage forms on the same GPU, against this line's FP32 lattice
        f16, l16, _ = single_lattice(lb, D, "couette4096_f16dev", args.steps, args.warmup, 0,
                                     reps=args.reps, target_s=args.target_s)
        l16.close()
        b16 = batch_measure(lb, D, "batch256_f16dev", args.steps, args.warmup, reps=5,
                            target_s=args.target_s)
        extra = {"couette4096_f16dev": f16, "batch256_f16dev": b16,
                 "batched_f16dev_over_f32_single": b16["mlups"] / value,
                 "single_f16dev_over_f32_single": f16["mlups"] / value}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cs = args.cpu_steps
        mlups_cpu, dt_cpu, cores = cpu_baseline_run(nx, ny, boundary, U, cs)
        cpu = {"value": mlups_cpu, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle, full {nx}x{ny} lattice of this workload, {cs} steps "
                         f"({dt_cpu:.1f} s), OpenMP {cores} threads"}
    if rank == 0:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "bytes_per_site": bytes_per_site,
                "peak_kind": peak_kind}
        if tr:
            roof["traffic_read"] = float(tr["read_bytes"])
            roof["traffic_write"] = float(tr["write_bytes"])
            roof["read_amplification"] = float(tr["read_bytes"]) / (bytes_per_site / 2 * sites)
            roof["traffic_source"] = tr.get("source")
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if storage != 0 else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "nx": nx, "ny": ny,
                           "boundary": "couette" if boundary else "periodic", "U_wall": U,
                           "storage": STORAGE_NAME[storage], "init": "bernoulli(0.7) droplets",
                           "l2": f"inputs larger than L2 ({lb.lb_state_bytes(nx, ny, storage) / 1e9:.2f} GB per buffer)",
                           "timing": f"median of {res['blocks']} timed blocks of {args.steps} "
                                     "graph-replayed steps, each between barriers",
                           "parallelism": f"replicas{world}",
                           "row_shape": res["row_shape"],
                           "row_shape_choice": ("timed at lb_create (lb_autotune, 8 steps "
                                                "per candidate)")
                           if storage == 1 and sites >= 1 << 22 else "default"},
                "roofline": roof,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "MLUPS",
                        "h2d_bytes_per_step": 18 * 2 * sites * es / args.steps,
                        "d2h_bytes_per_step": 7 * 8 / args.steps},
                "gpu_launches": args.steps * res["blocks"],
                "clocks": clocks_d,
                "reduced_storage": extra,
                "status": lb.lb_strerror(status),
                "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def run_mix(args):
    """An N_s = 3 species mixture (Sec. II for s = 1..N_s): MLUPS (site updates
    of all three species per second) as the median over repeated blocks of
    graph-free steps, against the bytes of 27 populations read and written."""
    import torch

    from paper_0906_3611_gb300 import lb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    nx, ny, storage = MIXES[args.workload]
    m = MIX3
    p = lb.make_mix_params(m["ns"], m["tau"], m["rho0"], m["Ga"], m["Gr"], m["G"],
                           storage=storage)
    stream = torch.cuda.Stream()
    mx = lb.Mixture(nx, ny, p, stream=stream)
    mx.init_random(rank, *MIX3_INIT)
    mass0 = mx.observables()["mass"]
    clocks = NvmlClocks(local)
    clocks.start()
    mx.step(args.warmup)
    mx.sync()
    ms = timed_blocks(D, stream, lambda: mx.step(args.steps), args.reps, clocks, args.target_s)
    clocks_d = clocks.stop()
    med = statistics.median(ms)
    mass1 = mx.observables()["mass"]
    status = mx.status()
    mx.close()
    sites = nx * ny
    value = whole_job_mlups(D.sum(sites * args.steps), med * 1e-3)
    bps = 2 * 9 * m["ns"] * ELEM[storage]
    peak, peak_kind = peaks()
    achieved = bps * sites / (med * 1e-3 / args.steps) / 1e9
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": med / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": STORAGE_NAME[storage], "data": "synthetic",
                "config": {"workload": args.workload, "nx": nx, "ny": ny, "species": m["ns"],
                           "boundary": "periodic", "storage": STORAGE_NAME[storage],
                           "couplings": "A/B emulsion set + dilute C, G_AC = G_BC = 0.2",
                           "timing": f"median of {len(ms)} timed blocks of {args.steps} steps",
                           "l2": f"inputs larger than L2 ({bps // 2 * sites / 1e9:.2f} GB per buffer)"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "bytes_per_site": bps,
                             "peak_kind": peak_kind},
                "mass_drift": float(max(abs(mass1 / mass0 - 1))),
                "gpu_launches": args.steps * len(ms), "clocks": clocks_d,
                "status": lb.lb_strerror(status), "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def run_sweep(args):
    """C3 at the Couette workload's size: every storage and wall speed, MLUPS and
    the FP64 stresses (mean sigma_xy, both walls) averaged over the second half
    of the run (sampled every `--sample-every` steps)."""
    import numpy as np
    import torch

    from paper_0906_3611_gb300 import lb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    rows = []
    every = max(1, args.sample_every)
    for name in ("couette4096_f32", "couette4096_f16dev", "couette4096_bf16dev"):
        nx, ny, boundary, _, storage = WORKLOADS[name]
        for U in (0.005, 0.02, 0.05):
            stream = torch.cuda.Stream()
            lat = lb.Lattice(nx, ny, lattice_params(lb, storage, boundary, U), stream=stream)
            lat.init_random(rank)
            lat.step(args.warmup)
            lat.sync()
            ms_total, acc, n_acc, t = 0.0, np.zeros(3), 0, 0
            while t < args.steps:
                k = min(every, args.steps - t)
                ms_total += timed_blocks(D, stream, lambda: lat.step(k), 1)[0]
                t += k
                if t > args.steps // 2:
                    acc += lat.observables()["stress"]
                    n_acc += 1
            st = lat.status()
            ob = lat.observables()
            lat.close()
            rows.append({"workload": name, "storage": STORAGE_NAME[storage], "U": U,
                         "mlups": whole_job_mlups(D.sum(nx * ny * args.steps), ms_total * 1e-3),
                         "stress_mean_second_half": (acc / max(n_acc, 1)).tolist(),
                         "stress_final": ob["stress"].tolist(), "mass_final": ob["mass"].tolist(),
                         "status": lb.lb_strerror(st)})
    if rank == 0:
        line = {"metric": "MLUPS", "value": statistics.median(r["mlups"] for r in rows),
                "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "couette4096_sweep", "nx": 4096, "ny": 4096,
                           "U_wall": [0.005, 0.02, 0.05], "storages": ["f32", "f16dev", "bf16dev"],
                           "stress": "[mean sigma_xy, wall_top, wall_bottom], FP64 reductions"},
                "sweep": rows, "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def batch_replicas(name):
    """The ensemble of a batch workload: sides uniform from the choices, Couette
    walls at U ~ U[0, Umax], seeds 0..n-1 (numpy Philox stream, seed 0)."""
    import numpy as np
    n, sides, umax, storage = BATCHES[name]
    g = np.random.Generator(np.random.Philox(key=0))
    side = g.choice(np.array(sides), size=n)
    U = g.uniform(0.0, umax, size=n)
    return [(int(side[k]), float(U[k]), k) for k in range(n)], storage


def batch_measure(lb, D, name, steps, warmup, reps=5, target_s=None, clocks=None):
    """A batched ensemble: all replicas in one persistent launch per step (the
    median over repeated blocks of `steps` graph-replayed launches), against the
    same replicas stepped one lattice at a time (sequential launches)."""
    import torch

    reps_list, storage = batch_replicas(name)
    stream = torch.cuda.Stream()

    def prm(U):
        return lb.make_params(**PHYS, boundary=lb.LB_COUETTE, U_wall=U, storage=storage,
                              rho_ref=(0.88, 0.44), init_kind=lb.LB_INIT_BERNOULLI, init=INIT)

    sites = sum(side * side for side, _, _ in reps_list)
    b = lb.Batch(len(reps_list), storage, stream)
    budget = 1 << 40  # effectively unbounded: every replica steps in every launch
    for side, U, seed in reps_list:
        b.add(side, side, prm(U), seed, budget)
    layout, rows = b.autotune(6)  # (6 timed steps per candidate: two were within noise)
    b.run(warmup)
    stream.synchronize()
    ms = timed_blocks(D, stream, lambda: b.run(steps), reps, clocks, target_s)
    status = b.status()
    b.close()
    med = statistics.median(ms)
    value = whole_job_mlups(D.sum(sites * steps), med * 1e-3)

    # the same replicas, one lattice at a time (each replica's steps in one lb_step)
    seq_steps = max(1, steps // 4)
    t_seq = 0.0
    for side, U, seed in reps_list:
        lat = lb.Lattice(side, side, prm(U), stream=stream).init_random(seed)
        lat.step(3)
        stream.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        lat.step(seq_steps)
        s1.record(stream)
        s1.synchronize()
        t_seq += s0.elapsed_time(s1)
        lat.close()
    seq_value = whole_job_mlups(D.sum(sites * seq_steps), D.max(t_seq) * 1e-3)
    es = ELEM[storage]
    bps = 2 * 18 * es
    peak, peak_kind = peaks()
    achieved = bps * sites / (med * 1e-3 / steps) / 1e9
    return {"workload": name, "mlups": value, "ms_per_step": med / steps, "blocks": len(ms),
            "steps_per_block": steps, "replicas": len(reps_list), "sites": sites,
            "sequential_single_lattice_mlups": seq_value, "over_sequential": value / seq_value,
            "work_list": {"layout": ["contiguous", "packed", "waves"][layout],
                          "max_piece_rows": rows},
            "bytes_per_site": bps, "achieved_gbs": achieved, "frac": achieved / peak,
            "peak_gbs": peak, "peak_kind": peak_kind, "storage": STORAGE_NAME[storage],
            "status": lb.lb_strerror(status)}


def run_batch(args):
    """Batched ensemble: all replicas in one persistent launch per step, against
    the same replicas stepped one lattice at a time (sequential launches)."""
    import torch

    from paper_0906_3611_gb300 import lb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    clocks = NvmlClocks(local)
    clocks.start()
    r = batch_measure(lb, D, args.workload, args.steps, args.warmup, reps=max(3, args.reps // 5),
                      target_s=args.target_s, clocks=clocks)
    clocks_d = clocks.stop()
    if rank == 0:
        line = {"metric": "MLUPS", "value": r["mlups"], "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "replicas": r["replicas"], "sites": r["sites"],
                           "sides": sorted(set(s for s, _, _ in batch_replicas(args.workload)[0])),
                           "storage": r["storage"], "boundary": "couette",
                           "U_wall": "uniform[0, 0.05]", "work_list": r["work_list"],
                           "timing": f"median of {r['blocks']} timed blocks of {args.steps} launches",
                           "l2": f"inputs larger than L2 ({r['sites'] * 18 * ELEM[BATCHES[args.workload][3]] / 1e9:.1f} GB per buffer set)"},
                "roofline": {"bound": "hbm", "achieved": r["achieved_gbs"], "peak": r["peak_gbs"],
                             "unit": "GB/s", "frac": r["frac"], "traffic": None,
                             "bytes_per_site": r["bytes_per_site"], "peak_kind": r["peak_kind"]},
                "sequential_single_lattice_mlups": r["sequential_single_lattice_mlups"],
                "gpu_launches": args.steps * r["blocks"], "clocks": clocks_d,
                "status": r["status"], "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def run_shear(args):
    """Ensemble of Kolmogorov-sheared lattices in one batch; the response R = U_k / U0
    of every replica after the timed steps gives the ensemble mean and kurtosis."""
    import numpy as np
    import torch

    from paper_0906_3611_gb300 import lb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    n, side, U0, storage = SHEARS[args.workload]
    nu, k = (STD07["tau"][0] - 0.5) / 3.0, 2.0 * np.pi / side
    g = U0 * nu * k * k
    stream = torch.cuda.Stream()
    p = lb.make_params(**STD07, storage=storage, rho_ref=(0.612, 0.612),
                       init_kind=lb.LB_INIT_UNIFORM_NOISE, init=(0.612, 0.612, 0.01),
                       g_kolmo=g, k_kolmo=1)
    b = lb.Batch(n, storage, stream)
    for r in range(n):
        b.add(side, side, p, 1000 * rank + r, args.warmup + args.steps + 64)
    layout, rows = b.autotune(2)
    for r in range(n):
        b.set_steps(r, args.warmup + args.steps)
    sampler = NvmlClocks(local)
    sampler.start()
    b.run(args.warmup)
    stream.synchronize()
    for r in range(n):  # the ageing snapshot phi(t_w) at t_w = warmup
        b.phi_snapshot(r)
    for r in range(n):  # U_k of every timed step, recorded on the device
        b.series_start(r, args.steps)
    D.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    sampler.loaded = True
    start.record(stream)
    b.run(args.steps)
    end.record(stream)
    end.synchronize()
    sampler.loaded = False
    D.barrier()
    clocks = sampler.stop()
    ms = start.elapsed_time(end)
    status = b.status()
    diag = [b.shear_diagnostics(r) for r in range(n)]
    ov = [b.phi_overlap(r) for r in range(n)]
    series = np.array([b.series(r) for r in range(n)]) / U0  # R(t) per replica
    nb = 24
    bursts = [b.series_bursts(r, 3.0, nb) for r in range(n)]
    b.close()
    # ensemble kurtosis K(t) = <R^4>/<R^2>^2 over the replicas at each recorded step (Fig. 16)
    Kt = np.mean(series ** 4, axis=0) / np.mean(series ** 2, axis=0) ** 2
    hist = np.sum([x["hist"] for x in bursts], axis=0)
    events = int(sum(x["events"] for x in bursts))
    # exponent of the burst-wait pdf (Fig. 14): least-squares slope of the
    # log-binned density over the bins holding at least 5 waits
    dens = hist / 2.0 ** np.arange(nb)
    used = hist >= 5
    alpha = (float(-np.polyfit(np.arange(nb)[used] + np.log2(1.5), np.log2(dens[used]), 1)[0])
             if used.sum() >= 3 else None)
    # R at three close late times over the ensemble (Fig. 17)
    late = series[:, -3:].ravel()
    late_sd = float(late.std())
    C = D.sum(sum(o[0] for o in ov)) / D.sum(sum(o[1] for o in ov))
    R = np.array(D.gather([d["U_k"] / U0 for d in diag]))
    iab = np.array(D.gather([d["I_AB"] for d in diag]))
    sites = n * side * side
    ms_max = D.max(ms)
    value = whole_job_mlups(D.sum(sites * args.steps), ms_max * 1e-3)
    es = ELEM[storage]
    achieved = 2 * 18 * es * sites / (ms * 1e-3 / args.steps) / 1e9
    peak, peak_kind = peaks()
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "replicas": n, "side": side,
                           "couplings": "rho0 = 0.7 standard set", "U0": U0, "g_kolmo": g,
                           "storage": STORAGE_NAME[storage],
                           "record": "U_k of every timed step, per replica, on the device",
                           "work_list": {"layout": ["contiguous", "packed", "waves"][layout],
                                         "max_piece_rows": rows},
                           "l2": f"{sites * 18 * es / 1e6:.0f} MB read per step: partly "
                                 "L2-resident (129 MB L2); not a bandwidth headline"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None,
                             "bytes_per_site": 2 * 18 * es, "peak_kind": peak_kind},
                "response": {"t": args.warmup + args.steps, "R_mean": float(R.mean()),
                             "R_kurtosis": float(np.mean(R ** 4) / np.mean(R ** 2) ** 2),
                             "I_AB_mean": float(iab.mean()),
                             "overlap_C": {"t_w": args.warmup, "dt_w": args.steps, "C": C},
                             "kurtosis_t": {"recorded_steps": int(Kt.size),
                                            "final": float(Kt[-1]), "mean": float(Kt.mean()),
                                            "max": float(Kt.max())},
                             "bursts": {"c_sigma": 3.0, "events": events,
                                        "wait_hist_log2": [int(v) for v in hist],
                                        "alpha_logbinned": alpha},
                             "R_late": {"samples": int(late.size), "mean": float(late.mean()),
                                        "sd": late_sd,
                                        "skew": float(np.mean((late - late.mean()) ** 3))
                                        / late_sd ** 3 if late_sd > 0 else None}},
                "gpu_launches": args.steps, "clocks": clocks,
                "status": lb.lb_strerror(status), "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def run_serve(args):
    """Serving loop: Poisson arrivals of simulation requests, continuous batching."""
    import numpy as np
    import torch

    from paper_0906_3611_gb300 import lb, serve

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    D = Dist()
    storage, n, rate, sides, steps_range, budget, slots, chunk = SERVES[args.workload]
    if args.requests:
        n = args.requests
    reqs = serve.poisson_requests(n, rate=rate, seed=rank, sides=sides, steps_range=steps_range)
    offered = sum(r.side * r.side * r.steps for r in reqs)
    srv = serve.Server(PHYS, storage, capacity=slots, chunk=chunk, budget_bytes=budget)
    sampler = NvmlClocks(local)
    sampler.start()
    D.barrier()
    t0 = time.perf_counter()
    sampler.loaded = True
    res = srv.run(reqs)
    torch.cuda.synchronize()
    sampler.loaded = False
    wall = time.perf_counter() - t0
    D.barrier()
    clocks = sampler.stop()
    srv.close()
    lat = np.array(D.gather([r.latency for r in res]))
    done_updates = D.sum(sum(r.side * r.side * r.steps for r in res))
    wall = D.max(wall)
    value = whole_job_mlups(done_updates, wall)
    offered = D.sum(offered)
    completed = int(D.sum(len(res)))
    span = D.max(max(r.arrival for r in reqs))
    steps_done = int(D.sum(sum(r.steps for r in res)))
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": steps_done, "warmup": 0,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "requests": n, "arrival_rate_per_s": rate,
                           "sides": f"uniform {sides[0]}..{sides[-1]} step 64",
                           "steps": "log-uniform [1e3, 1e5]", "hbm_budget_gb": budget / 1e9,
                           "slots": slots, "chunk_steps": chunk, "storage": STORAGE_NAME[storage]},
                "served": {"completed": completed, "wall_s": wall,
                           "latency_p50_s": float(np.percentile(lat, 50)),
                           "latency_p99_s": float(np.percentile(lat, 99)),
                           "offered_mlups": offered / max(span, 1e-9) / 1e6,
                           "overload_factor": (offered / max(span, 1e-9)) / (done_updates / wall)},
                "clocks": clocks, "impl": "gb300"}
        print(json.dumps(line), flush=True)
    D.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="couette4096_f32",
                    choices=sorted(WORKLOADS) + sorted(BATCHES) + sorted(SHEARS) + sorted(SERVES)
                    + sorted(MIXES) + ["couette4096_sweep"])
    ap.add_argument("--requests", type=int, default=0)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the reduced-storage keys of the default line")
    ap.add_argument("--reps", type=int, default=25, help="timed blocks of --steps steps (minimum)")
    ap.add_argument("--target-s", type=float, default=1.5,
                    help="grow the timed blocks to about this many seconds")
    ap.add_argument("--sample-every", type=int, default=1000,
                    help="couette4096_sweep: steps between stress samples")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "couette4096_sweep":
        run_sweep(args)
    elif args.workload in MIXES:
        run_mix(args)
    elif args.workload in BATCHES:
        run_batch(args)
    elif args.workload in SHEARS:
        run_shear(args)
    elif args.workload in SERVES:
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
