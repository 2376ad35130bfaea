"""Benchmark: saturated vs as-written FP64 compressible-flow RHS at 256^3 on GB300.

One step = one call of `acs_rhs_saturated` over the 256^3 interior (+2 halo) of the
seeded synthetic field, inputs resident in HBM (703 MB in + 671 MB out, both larger than
the 129 MB L2, so no flush is needed between steps). The as-written form
(`acs_rhs_plain`) is timed on the same input in the same run, and so are both forms of the
25-point star stencil at 384^3, as context.

Printed: one JSON line (rank 0). `value` = Gpoint-updates/s of the saturated form summed
over ranks (each rank runs its own replica: no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gpoint-updates/s & HBM GB/s, saturated vs as-written, 256^3 FP64, ≤1e-12 rel"
UNIT = "Gpoint-updates/s"
N_RHS = 256
N_STAR = 384

# FP64-pipe operations per interior point of the saturated RHS, from its expression DAG
# (FMA, add, mul each one pipe operation). With three spacings: per point 21 for the fluxes
# (3 Newton FMAs of the reciprocal, 3 velocities, 2 for |m.v|, 2 for P, E+P, 3 diagonal,
# 3 off-diagonal, 3 energy) + 5 components x 19 (3 differences, 3 for the scaled flux sum,
# 10 for S2 and S1, 2 for S2 - 4 S1 + 18 U, 1 final FMA) = 116; the rewriter's march variants
# compute this form. With equal spacing (the benchmark grids) the built-in kernel folds
# -1/(2h) into the fluxes: 23 for the fluxes (+ the scaled reciprocal and pressure) + 19 for
# the mass component + 4 x 18 (2 adds in place of 3 scaled terms) = 114.
# The star stencil: 1 + 12 x 2 + 1 = 26.
DP_OPS_PER_POINT = {"rhs_saturated": 114, "rhs_saturated_anisotropic": 116, "star_saturated": 26}
# The FP64 pipe's nominal issue rate: 2 operations / clock / SM (nominal 1.25 TFLOP/s of FMA
# at 2070 MHz on 152 SMs: 1.25e12 / 2 / 152 / 2.07e9 = 1.99). The roofline's peak is the rate
# the FP64 probe measures in the same run; 2 x SMs x max SM clock (both queried from the device)
# is reported beside it as the derived peak. The constants are used only when a query fails.
DP_OPS_PER_CLK_SM = 2
FALLBACK_SMS = 152
FALLBACK_SM_MAX_MHZ = 2070.0

# DRAM bytes per launch measured by ncu, keyed by the SHA-256 of the files that define the
# kernel and by the launch shape; a changed kernel or another shape reports null until it is
# profiled again.
NCU_TRAFFIC = {
    # one-pass ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of one launch at
    # 256^3, the 4th after 3 warm-ups, in the shapes the autotuner picks
    "cd1a3ed280707f36:16x16, balanced, TMA": 830774016 + 633936384,
    "cd1a3ed280707f36:32x8, balanced, TMA": 858266368 + 633995520,
}


def kernel_source_hash() -> str:
    """Hash of the code (comments and whitespace removed) the saturated RHS kernel is compiled
    from: rhs_saturated.cu, device_ops.cuh, tma.cuh and the RHS part of march.cuh (everything
    before the star stencil's StarShape). A comment edit, or an edit of the star stencil's
    march, keeps the recorded ncu traffic; a code edit of the RHS kernel drops it."""
    import re
    h = hashlib.sha256()
    for f in ("march.cuh", "rhs_saturated.cu", "device_ops.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_2306_13002_gb300", "csrc", f)) as fh:
            text = fh.read()
        if f == "march.cuh":
            text = text[:text.index("struct StarShape")]
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver): SM clock,
    maximum SM clock, power and the active clock-event reasons. Nothing is set."""

    CLOCK_SM = 1
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int = 0):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        ok = False
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(cuda_index)
            if hasattr(pr, "pci_bus_id"):
                bus = "%08x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), pr.pci_bus_id,
                                            getattr(pr, "pci_device_id", 0))
        except Exception:
            bus = None
        if bus is not None:
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.dev)) == 0
        if not ok:
            visible = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            idx = cuda_index
            if visible and visible.split(",")[cuda_index].strip().isdigit():
                idx = int(visible.split(",")[cuda_index])
            if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(self.dev)) != 0:
                raise RuntimeError("no NVML handle for the device")
        self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _uint(self, fn, *args) -> int | None:
        v = self.ct.c_uint()
        return int(v.value) if fn(self.dev, *args, self.ct.byref(v)) == 0 else None

    def sm_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, self.ct.c_int(self.CLOCK_SM))

    def sm_max_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, self.ct.c_int(self.CLOCK_SM))

    def power_w(self):
        mw = self._uint(self.lib.nvmlDeviceGetPowerUsage)
        return None if mw is None else mw / 1000.0

    def reasons(self):
        v = self.ct.c_ulonglong()
        if self._reasons(self.dev, self.ct.byref(v)) != 0:
            return None
        return sorted(name for bit, name in self.REASONS.items() if v.value & bit)


class ClockSampler:
    """Samples the SM clock, power and clock-event reasons every `period_s` (in-process NVML,
    else `nvidia-smi -lms 100`) while the bench runs; `summary` keeps the samples that fall in
    the timed windows registered with `window(t0, t1)`."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_s: float = 0.004):
        self.gpu = gpu_index
        self.period = period_s
        self.samples = []          # (time, sm_mhz, max_mhz, power_w, [reasons])
        self.windows = []
        self.proc = None
        self.thread = None
        self.stop_flag = threading.Event()
        self.paused = threading.Event()
        self.source = None
        try:
            self.nvml = Nvml(gpu_index)
            self.max_mhz = self.nvml.sm_max_mhz()
        except Exception:
            self.nvml = None
            self.max_mhz = None

    def start(self):
        if self.nvml is not None:
            self.source = f"NVML in-process, every {self.period * 1e3:.0f} ms"
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.source = "nvidia-smi -lms 100"
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _poll(self):
        while not self.stop_flag.is_set():
            t = time.time()
            if not self.paused.is_set():
                try:
                    self.samples.append((t, self.nvml.sm_mhz(), self.max_mhz, self.nvml.power_w(),
                                         self.nvml.reasons()))
                except Exception:
                    pass
            self.stop_flag.wait(self.period)

    def pause(self):
        """Stop querying NVML until resume() (in-process sampling only). Used around the e2e leg:
        with the queries running, steps of the host-streamed pipeline were slow more often (7
        against 2 in 300 steps, by 0.5-0.9 ms), as if the queries delayed the pipeline's own
        calls into the driver."""
        self.paused.set()

    def resume(self):
        self.paused.clear()

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            r = [x.strip() for x in line.split(",")]
            if len(r) < 9:
                continue
            num = lambda v: float(v) if v.replace(".", "").isdigit() else None  # noqa: E731
            self.samples.append((time.time(), num(r[1]), num(r[2]), num(r[3]),
                                 [n for n, v in zip(names, r[5:9]) if v.lower() == "active"]))

    def window(self, t0: float, t1: float):
        self.windows.append((t0, t1))

    def stop(self):
        self.stop_flag.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def median_mhz(self, t0: float, t1: float):
        sm = [r[1] for r in self.samples if t0 <= r[0] <= t1 and r[1]]
        return statistics.median(sm) if sm else None

    def summary(self) -> dict:
        rows = [r for r in self.samples if any(a <= r[0] <= b for a, b in self.windows)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no clock samples"], "samples": 0,
                    "source": self.source}
        sm = [r[1] for r in rows if r[1]]
        mx = [r[2] for r in rows if r[2]] or ([self.max_mhz] if self.max_mhz else [])
        pw = [r[3] for r in rows if r[3] is not None]
        reasons = sorted({n for r in rows for n in (r[4] or [])})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_min_mhz": min(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None, "timed_windows": len(self.windows),
                "source": self.source}


def tile_text(tile) -> str:
    """'32x8, z-chunk 16' or '16x16, balanced, TMA' for an (bx, by, kchunk[, flags]) tuple."""
    from paper_2306_13002_gb300 import binding
    bx, by, kc, flags = (tuple(tile) + (0, 0, 0, 0))[:4]
    text = f"{bx}x{by}, " + ("balanced" if flags & binding.TILE_BALANCED else f"z-chunk {kc}")
    return text + (", TMA" if flags & binding.TILE_TMA else "")


def cpu_baseline(U: np.ndarray, budget_s: float = 10.0) -> dict:
    """The oracle (as-written FP64 loop nest, gcc) on a bounded z-slab sample of the same field."""
    import oracle
    threads = os.cpu_count() or 1
    if not oracle.has_openmp():
        threads = 1
    n = U.shape[-1] - 4
    out = np.empty((5, n, n, n))            # one output array for every call: the timing is the oracle's
    out.fill(0.0)
    passes, pts, dt = 0, 0, 0.0
    while dt < budget_s and passes < 200:      # whole-field passes until ~budget_s of wall time
        t = time.perf_counter()
        oracle.rhs(U, threads=threads, out=out)
        dt += time.perf_counter() - t
        pts += n ** 3
        passes += 1
    # the same oracle on one thread, one call over about 2 s worth of whole z-planes (sized from a
    # 4-plane call)
    one = {"value": None, "planes": 0}
    if threads > 1:
        t = time.perf_counter()
        oracle.rhs(U, k_range=(0, min(4, n)), threads=1, out=out)
        t4 = time.perf_counter() - t
        planes = int(max(1, min(n, 4 * 2.0 / max(t4, 1e-3))))
        t = time.perf_counter()
        oracle.rhs(U, k_range=(0, planes), threads=1, out=out)
        one = {"value": planes * n * n / (time.perf_counter() - t) / 1e9, "planes": planes}
    return {"value": pts / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"as-written RHS oracle, {passes} passes over the whole {n}^3 field ({pts} points, {dt:.1f} s)",
            "host_cpu": cpu_model(), "single_thread_value": one["value"],
            "single_thread_sample": f"{one['planes']} z-planes of the same field on one core"}


def cpu_model() -> str:
    """The host CPU as the OS names it (model name, or the implementer and part on Arm)."""
    import platform
    name, impl, part = None, None, None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip().lower(), v.strip()
                if k == "model name" and not name:
                    name = v
                elif k == "cpu implementer" and not impl:
                    impl = v
                elif k == "cpu part" and not part:
                    part = v
    except OSError:
        pass
    if name:
        return f"{name} ({platform.machine()})"
    if impl or part:
        return f"{platform.machine()} implementer {impl} part {part}"
    return platform.machine() or "unknown"


def run_reference(args) -> None:
    """Reference arm: the CPU oracle, as it stands, on host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2306_13002_gb300 import inputs
    oracle.build()
    U = inputs.rhs_field(N_RHS, halo=2, seed=inputs.SEED_RHS_LARGE)
    threads = os.cpu_count() or 1
    if not oracle.has_openmp():
        threads = 1
    out = np.empty((5, N_RHS, N_RHS, N_RHS))   # one output array for every call, its pages touched once
    out.fill(0.0)
    oracle.rhs(U, k_range=(0, 1), threads=threads, out=out)   # thread pool start-up
    t = time.perf_counter()
    oracle.rhs(U, k_range=(0, 4), threads=threads, out=out)
    t1 = max((time.perf_counter() - t) / 4, 1e-5)             # per plane
    total = max(1, args.steps + args.warmup)
    planes = int(max(1, min(N_RHS, 120.0 / total / t1)))
    times = []
    for s in range(total):
        k0 = (s * planes) % (N_RHS - planes + 1)
        t = time.perf_counter()
        oracle.rhs(U, k_range=(k0, k0 + planes), threads=threads, out=out)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
    pts = planes * N_RHS * N_RHS
    mean = sum(times) / len(times)
    value = pts / mean / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(N_RHS, args.gpus),
        "form": "as written, the CPU oracle (plain C, FP64, no FMA contraction)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{planes} z-planes of the {N_RHS}^3 field per step ({pts} points)",
                         "host_cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def workload_config(n: int, world: int) -> dict:
    """The workload both arms run (the same dict in the reference arm's line): the RHS of the
    compressible Euler equations with 4th-order dissipation on an n^3 grid, FP64."""
    in_b, out_b = 5 * (n + 4) ** 3 * 8, 5 * n ** 3 * 8
    return {"workload": f"rhs_{n}^3_fp64", "grid": [n] * 3, "halo": 2, "gamma": 1.4, "eps": 0.25,
            "h": [1.0, 1.0, 1.0], "l2": f"inputs larger than L2 ({in_b / 1e6:.0f} MB in, {out_b / 1e6:.0f} MB out)",
            "parallelism": f"replicas x{world}"}


def reduce_over_ranks(dist, x: float, op: str, device: str) -> float:
    """Max or sum of a per-rank scalar over all ranks (identity without a process group).

    Used only for timing and throughput bookkeeping: the replicas exchange no data."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(dist, region_ms_local: float, steps: int, points_local: float, device: str):
    """Weak-scaling bookkeeping of independent replicas: the job's time per step is the slowest
    rank's (max over ranks) and its throughput the points of all ranks over that time.
    Returns (ms per step, Gpoint-updates/s of the job, points of the job per step)."""
    ms = reduce_over_ranks(dist, region_ms_local, "max", device) / steps
    pts = reduce_over_ranks(dist, float(points_local), "sum", device)
    return ms, pts / (ms * 1e-3) / 1e9, pts


def wall_timer(fn, steps: int) -> float:
    """Host wall-clock time of `steps` calls (ms); the timer of the CPU replicas."""
    t = time.perf_counter()
    for _ in range(steps):
        fn()
    return (time.perf_counter() - t) * 1e3


def timed_replica_region(dist, fn, steps: int, timer, sync=lambda: None) -> float:
    """One rank's timed region: barrier, sync, `steps` calls timed by `timer` (ms), sync,
    barrier. Returns this rank's region time in ms."""
    if dist:
        dist.barrier()
    sync()
    ms = timer(fn, steps)
    sync()
    if dist:
        dist.barrier()
    return ms


def launch_plan(gpus: int, env) -> str:
    """'run' when this process is the whole job or one of `gpus` ranks, 'relaunch' when one
    process was started for several GPUs (bench.py starts torchrun itself), else an error."""
    if "WORLD_SIZE" in env:
        ws = int(env["WORLD_SIZE"])
        if ws != gpus:
            return f"error: --gpus {gpus} but WORLD_SIZE={ws}"
        return "run"
    return "relaunch" if gpus > 1 else "run"


def relaunch(args_list, gpus: int) -> int:
    """Run this script under torch.distributed.run with one rank per GPU (127.0.0.1 rendezvous);
    returns its exit code. Rank 0 prints the JSON line."""
    import socket
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *args_list]
    return subprocess.call(cmd)


def fp64_probe(torch, binding, stream, sms: int, sampler, blocks_per_sm: int = 2, threads: int = 256,
               iters: int = 8192, reps: int = 5) -> dict:
    """The FP64 pipe's measured rate (acs_fp64_rate_probe: register-only FMA chains) at the RHS
    kernel's occupancy (2 blocks of 256 threads per SM), timed with CUDA events."""
    sink = torch.empty(sms * blocks_per_sm * threads, dtype=torch.float64, device="cuda")
    run = lambda: binding.acs_fp64_rate_probe(sink, sms * blocks_per_sm, threads, iters, stream=stream)  # noqa: E731
    ops = run()
    run()
    torch.cuda.synchronize()
    t0 = time.time()
    launch_ms, _ = time_launches(torch, run, reps, stream)
    t1 = time.time()
    if sampler:
        sampler.window(t0, t1)
    gops = ops / (launch_ms * 1e-3) / 1e9
    mhz = sampler.median_mhz(t0, t1) if sampler else None
    return {"gops": gops, "op_per_clk_per_sm": gops * 1e3 / (mhz * sms) if mhz else None, "sm_mhz": mhz,
            "blocks_per_sm": blocks_per_sm, "threads": threads, "ops_per_launch": ops, "launch_ms": launch_ms}


def host_link_floor(torch, U_pin, U, R, R_pin, stream, reps: int) -> dict:
    """The host link under the end-to-end step, measured on the same pinned buffers: the upload of
    U alone, the download of R alone, and both at once on two streams (the floor of a step that
    moves both, whatever the overlap with the kernel)."""
    side = torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def both():
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            R_pin.copy_(R, non_blocking=True)
        U.copy_(U_pin, non_blocking=True)
        stream.wait_stream(side)

    up = timed(lambda: U.copy_(U_pin, non_blocking=True))
    down = timed(lambda: R_pin.copy_(R, non_blocking=True))
    bi = timed(both)
    nu, nd = U.numel() * 8, R.numel() * 8
    return {"upload_ms": up, "download_ms": down, "both_ms": bi, "upload_gbs": nu / (up * 1e-3) / 1e9,
            "download_gbs": nd / (down * 1e-3) / 1e9, "both_gbs": (nu + nd) / (bi * 1e-3) / 1e9}


def time_launches(torch, fn, steps: int, stream, per=None) -> tuple[float, float]:
    """Per-launch CUDA-event durations on `stream`; returns (mean launch ms, region ms) and
    appends every launch's duration to `per` if given."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # no garbage collection while the steps are enqueued (as timeit does): a collection pause in
    # the enqueue loop would leave the GPU idle between steps and be timed as part of a step
    gc_on = gc.isenabled()
    gc.disable()
    try:
        r0.record(stream)
        for s in range(steps):
            starts[s].record(stream)
            fn()
            ends[s].record(stream)
        r1.record(stream)
        torch.cuda.synchronize()
    finally:
        if gc_on:
            gc.enable()
    durations = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    if per is not None:
        per.extend(durations)
    return sum(durations) / len(durations), r0.elapsed_time(r1)


def bench_block(torch, binding, inputs, stream, steps: int) -> dict:
    """The block-assembly body (75 statements, 151 loads per point) at 128^3, four forms."""
    n = 128
    A, B, G = inputs.block_fields(n, halo=1, seed=inputs.SEED_BLOCK)
    Ad, Bd, Gd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), torch.from_numpy(G).cuda()
    del A, B, G
    out = torch.empty((75, n, n, n), dtype=torch.float64, device="cuda")
    res = {"grid": [n] * 3, "bytes_per_point_algorithmic": 8 * (51 + 75)}
    for form in ("as_written", "cse", "cse_bulk", "saturated"):
        fn = lambda f=form: binding.acs_block_form(Ad, Bd, Gd, out, f, stream=stream)  # noqa: E731
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        _, rm = time_launches(torch, fn, steps, stream)
        ms = rm / steps
        res[form] = {"ms": ms, "gpts": n ** 3 / (ms * 1e-3) / 1e9,
                     "hbm_gbs_algorithmic": 8 * (51 + 75) * n ** 3 / (ms * 1e-3) / 1e9}
    del Ad, Bd, Gd, out
    torch.cuda.empty_cache()
    return res


def bench_batch(torch, binding, inputs, stream, steps: int, tile=None) -> dict:
    """64 star-stencil grids, sides log-uniform in [16, 160]: per-grid launches vs one
    persistent batch launch vs the autotuned batch replayed from a CUDA graph (`tile`: use this
    shape for both batch legs instead of the default and the autotuner's)."""
    given = tile is not None
    sides = inputs.batch_sides(64, seed=inputs.SEED_BATCH)

    def dev(arr):
        """Device copy with rows padded to an even pitch (whole 16-byte units), a layout tensor
        copies can stage; most sides are odd, so the unpadded pitch (side + 8) would be odd."""
        X = arr.shape[-1]
        if X % 2 == 0:
            return torch.from_numpy(arr).cuda()
        return torch.from_numpy(inputs.pad_rows(arr, X + 1).base).cuda()[..., :X]

    grids = []
    for q, (nx, ny, nz) in enumerate(sides):
        u, a = inputs.stencil_fields(int(nx), int(ny), int(nz), halo=4, seed=inputs.SEED_BATCH + 100 + q)
        grids.append((dev(u), dev(a), torch.empty((int(nz), int(ny), int(nx)), dtype=torch.float64, device="cuda")))
    points = int(sum(int(a) * int(b) * int(c) for a, b, c in sides))
    ws = torch.zeros((binding.acs_batch_workspace_bytes(64) + 15) // 16 * 2, dtype=torch.float64, device="cuda")
    res = {"grids": 64, "points": points, "layout": "input rows padded to an even pitch"}

    def per_grid():
        for (u, a, out) in grids:
            binding.acs_stencil_saturated(u, a, out, stream=stream)

    plan = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws, tile=tile, stream=stream)
    batch = lambda: binding.acs_batch_launch(plan, stream=stream)  # noqa: E731
    for name, fn in (("per_grid_launches", per_grid), ("batch_launch", batch)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        _, rm = time_launches(torch, fn, steps, stream)
        res[name] = {"ms": rm / steps, "gpts": points / (rm / steps * 1e-3) / 1e9}
    if tile is None:
        tile, _ = binding.acs_autotune_batch(binding.KIND_STENCIL, grids, ws, stream=stream)
    plan_t = binding.acs_batch_prepare(binding.KIND_STENCIL, grids, ws, tile=tile, stream=stream)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        binding.acs_batch_launch(plan_t, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        binding.acs_batch_launch(plan_t, stream=torch.cuda.current_stream())
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    _, rm = time_launches(torch, graph.replay, steps, stream)
    res["graph_autotuned"] = {"ms": rm / steps, "gpts": points / (rm / steps * 1e-3) / 1e9, "tile": list(tile),
                              "tile_source": "given" if given else "acs_autotune_batch"}
    return res


def bench_ranker(binding, ranker, n_variants: int = 512) -> dict:
    """The learned ranker on the saturated (march-scope) variants at 256^3: a study of the distinct
    ones among `n_variants` rewriter variants (78 % train, the rest ranked by the MLP and by the
    paper's analytical cost), every variant checked against the library's saturated kernel."""
    t = time.time()
    res = ranker.study(n_variants=n_variants, n=N_RHS, epochs=2000, reps=5, scope=binding.SCOPE_MARCH,
                       extra_splits=20, search_candidates=2048)
    res["wall_s"] = time.time() - t
    return res


def bench_large(torch, binding, inputs, stream, peak_gops: float, pick_index: int | None, steps: int) -> dict:
    """RHS 512^3 (as written, autotuned saturated, the ranker-picked saturated variant) and the star
    stencil at 768^3 (as written, autotuned saturated), with fractions of the FP64-pipe roofline
    (measured peak) and of HBM."""
    from paper_2306_13002_gb300 import ranker  # noqa: F401
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    out = {"fp64_peak_gops": peak_gops}
    n = 512
    U = torch.from_numpy(inputs.rhs_field(n, halo=2, seed=inputs.SEED_HUGE)).cuda()
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    pts = n ** 3
    algo_bytes = (U.numel() + R.numel()) * 8
    rhs = {"grid": [n] * 3, "in_gb": U.numel() * 8 / 1e9, "out_gb": R.numel() * 8 / 1e9}
    tile, _ = binding.acs_autotune_rhs(U, R, stream=stream)
    forms = [("as_written", lambda: binding.acs_rhs_plain(U, R, stream=stream)),
             ("saturated_autotuned", lambda: binding.acs_rhs_saturated(U, R, tile=tile, stream=stream))]
    pick = None
    if pick_index is not None:
        src, _, info = binding.acs_variant_generate(inputs.SEED_VARIANTS, pick_index, binding.SCOPE_MARCH)
        pick = binding.Variant(src, info)
        forms.append(("ranker_pick_variant", lambda: binding.acs_rhs_saturated(U, R, variant=pick, stream=stream)))
    for form, fn in forms:
        fn()
        torch.cuda.synchronize()
        _, rm = time_launches(torch, fn, steps, stream)
        ms = rm / steps
        rhs[form] = {"ms": ms, "gpts": pts / (ms * 1e-3) / 1e9}
    if pick is not None:
        rhs["ranker_pick_variant"].update({"index": pick_index, "shape": [*pick.block, pick.flags],
                                           "fp64_frac_at_116_ops": DP_OPS_PER_POINT["rhs_saturated_anisotropic"] * pts /
                                           (rhs["ranker_pick_variant"]["ms"] * 1e-3) / 1e9 / peak_gops})
        pick.close()
    sat = rhs["saturated_autotuned"]["ms"]
    rhs["tile"] = list(tile)
    rhs["fp64_frac"] = DP_OPS_PER_POINT["rhs_saturated"] * pts / (sat * 1e-3) / 1e9 / peak_gops
    rhs["hbm_frac"] = algo_bytes / (sat * 1e-3) / 1e9 / hbm
    rhs["speedup_saturated_over_as_written"] = rhs["as_written"]["ms"] / sat
    out["rhs_512"] = rhs
    del U, R
    torch.cuda.empty_cache()
    n = 768
    u_np, a_np = inputs.stencil_fields(n, halo=4, seed=inputs.SEED_HUGE)
    u, a = torch.from_numpy(u_np).cuda(), torch.from_numpy(a_np).cuda()
    del u_np, a_np
    o = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    pts = n ** 3
    algo_bytes = (u.numel() + a.numel() + o.numel()) * 8
    st = {"grid": [n] * 3}
    tile, _ = binding.acs_autotune_stencil(u, a, o, stream=stream)
    for form, fn in (("as_written", lambda: binding.acs_stencil_plain(u, a, o, stream=stream)),
                     ("saturated_autotuned", lambda: binding.acs_stencil_saturated(u, a, o, tile=tile, stream=stream))):
        fn()
        torch.cuda.synchronize()
        _, rm = time_launches(torch, fn, steps, stream)
        ms = rm / steps
        st[form] = {"ms": ms, "gpts": pts / (ms * 1e-3) / 1e9}
    sat = st["saturated_autotuned"]["ms"]
    st["tile"] = list(tile)
    st["fp64_frac"] = DP_OPS_PER_POINT["star_saturated"] * pts / (sat * 1e-3) / 1e9 / peak_gops
    st["hbm_frac"] = algo_bytes / (sat * 1e-3) / 1e9 / hbm
    st["speedup_saturated_over_as_written"] = st["as_written"]["ms"] / sat
    out["stencil_768"] = st
    del u, a, o
    torch.cuda.empty_cache()
    return out


def run_large(args) -> None:
    """--large alone: the ranker study (512 variants at 256^3), then the large workloads."""
    import torch
    from paper_2306_13002_gb300 import binding, inputs, ranker
    from paper_2306_13002_gb300 import build as acs_build
    acs_build.build()
    stream = torch.cuda.current_stream()
    sms = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    peak = fp64_probe(torch, binding, stream, sms, None)["gops"]
    study = bench_ranker(binding, ranker)
    res = bench_large(torch, binding, inputs, stream, peak, study["mlp_pick_index"], max(3, min(args.steps, 10)))
    print(json.dumps({"study": "large workloads", "unit": UNIT, "ranker_256": study, **res}))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stencil", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the as-written timing")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end timing")
    ap.add_argument("--no-ranker", action="store_true", help="skip the learned-ranker study (and the large block)")
    ap.add_argument("--no-large", action="store_true", help="skip RHS 512^3 and the star stencil at 768^3")
    ap.add_argument("--n", type=int, default=N_RHS, help="RHS interior side (256 is the benchmark workload)")
    ap.add_argument("--ranker", action="store_true",
                    help="instead of the step benchmark: the rewriter-variant ranker study (512 variants at 256^3)")
    ap.add_argument("--variants", type=int, default=512)
    ap.add_argument("--scope", default="march", choices=["march", "iteration"],
                    help="--ranker: rank cross-iteration saturated kernels (march) or per-point bodies")
    ap.add_argument("--tile", default="", help="bx,by,kchunk[,flags]: use this launch shape instead of the autotuner")
    ap.add_argument("--large", action="store_true",
                    help="instead of the step benchmark: RHS 512^3 and star stencil 768^3, all forms")
    ap.add_argument("--batch", action="store_true",
                    help="instead of the step benchmark: the 64-grid star-stencil batch alone")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.steps = max(args.steps, 1)
    if args.impl == "reference":
        run_reference(args)
        return
    plan = launch_plan(args.gpus, os.environ)
    if plan == "relaunch":
        sys.exit(relaunch(sys.argv[1:], args.gpus))
    if plan != "run":
        print(plan, file=sys.stderr)
        sys.exit(2)
    if args.large:
        run_large(args)
        return
    if args.batch:
        import torch
        from paper_2306_13002_gb300 import binding, inputs
        from paper_2306_13002_gb300 import build as acs_build
        acs_build.build()
        stream = torch.cuda.current_stream()
        tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
        res = bench_batch(torch, binding, inputs, stream, max(3, min(args.steps, 50)), tile=tile)
        print(json.dumps({"workload": "star_stencil_batch_64_grids_fp64", "unit": "ms per batch", **res}))
        return
    if args.ranker:
        from paper_2306_13002_gb300 import binding, ranker
        from paper_2306_13002_gb300 import build as acs_build
        acs_build.build()
        t = time.time()
        res = ranker.study(n_variants=args.variants, n=args.n,
                           scope=binding.SCOPE_ITERATION if args.scope == "iteration" else binding.SCOPE_MARCH)
        res["wall_s"] = time.time() - t
        print(json.dumps({"study": "learned variant ranker", "metric": "chosen-variant time / measured best",
                          "unit": "ratio", **res}))
        return
    run_ours(args)


def run_ours(args) -> None:
    """The step benchmark: one replica per rank (torchrun sets RANK / WORLD_SIZE)."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2306_13002_gb300 import binding, inputs
    from paper_2306_13002_gb300 import build as acs_build
    if rank == 0:
        acs_build.build()
    if dist:
        dist.barrier()
    binding.lib()
    sync = torch.cuda.synchronize
    props = torch.cuda.get_device_properties(local)
    sms = int(getattr(props, "multi_processor_count", 0)) or FALLBACK_SMS

    n = args.n
    U_host = inputs.rhs_field(n, halo=2, seed=inputs.SEED_RHS_LARGE + rank)
    U_pin = torch.from_numpy(U_host).pin_memory()
    R_pin = torch.empty((5, n, n, n), dtype=torch.float64).pin_memory()
    U = U_pin.to("cuda")
    R = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    points = n ** 3
    in_bytes = U.numel() * 8
    out_bytes = R.numel() * 8

    def timer(fn, steps):               # CUDA events on the launching stream
        return time_launches(torch, fn, steps, stream)[1]

    sat = lambda: binding.acs_rhs_saturated(U, R, stream=stream)  # noqa: E731
    plain = lambda: binding.acs_rhs_plain(U, R, stream=stream)  # noqa: E731

    # Launch shape from the library's autotuner (outside the timed region); tile=None calls
    # then use the tuned shape from the cache.
    if args.tile:
        tuned_tile = tuple(int(v) for v in args.tile.split(","))
        sat = lambda: binding.acs_rhs_saturated(U, R, tile=tuned_tile, stream=stream)  # noqa: E731
    else:
        tuned_tile, _ = binding.acs_autotune_rhs(U, R, stream=stream)
    for _ in range(args.warmup):
        sat()
    sync()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.2)
    # The FP64 pipe's measured rate, the roofline's denominator (same process, same clocks).
    probe = fp64_probe(torch, binding, stream, sms, sampler)

    if dist:
        dist.barrier()
    sync()
    t0 = time.time()
    launch_ms, region_ms = time_launches(torch, sat, args.steps, stream)
    t1 = time.time()
    sync()
    if dist:
        dist.barrier()
    if sampler:
        sampler.window(t0, t1)
    launch_ms = reduce_over_ranks(dist, launch_ms, "max", "cuda")
    ms_per_step, value, _ = replica_throughput(dist, region_ms, args.steps, points, "cuda")
    main_mhz = sampler.median_mhz(t0, t1) if sampler else None

    def timed(fn, steps):
        """(ms per step, job Gpoint/s) of a timed leg, its window registered with the sampler."""
        ta = time.time()
        rm = timed_replica_region(dist, fn, steps, timer, sync)
        if sampler:
            sampler.window(ta, time.time())
        ms, val, _ = replica_throughput(dist, rm, steps, points, "cuda")
        return ms, val

    # As-written form on the same input.
    as_written = None
    if not args.no_plain:
        for _ in range(2):
            plain()
        sync()
        plain_ms, plain_value = timed(plain, max(3, min(args.steps, 40)))
        as_written = {"value": plain_value, "ms_per_step": plain_ms,
                      "speedup_saturated_over_as_written": plain_ms / ms_per_step}

    # The paper's ablation ladder on the same input (Sec. VII code versions).
    ladder = None
    if not args.no_plain:
        ladder = {}
        for form in ("cse", "cse_sat", "cse_bulk", "accsat"):
            fn = lambda f=form: binding.acs_rhs_form(U, R, f, stream=stream)  # noqa: E731
            for _ in range(2):
                fn()
            sync()
            ms, val = timed(fn, max(3, min(args.steps, 40)))
            ladder[form] = {"ms": ms, "value": val}
        if as_written:
            ladder["as_written"] = {"ms": as_written["ms_per_step"], "value": as_written["value"]}
        ladder["saturated"] = {"ms": ms_per_step, "value": value}

    # End to end through the public API with host buffers: acs_rhs_saturated_host streams
    # pinned U through the GPU in z-slabs (upload, kernel and download overlapped) into pinned R.
    e2e = None
    if not args.no_e2e:
        ws_e2e = torch.empty(binding.acs_rhs_host_workspace_bytes(U_pin, R_pin) // 8 + 2, dtype=torch.float64,
                             device="cuda")
        e2e_step = lambda: binding.acs_rhs_saturated_host(U_pin, R_pin, ws_e2e, stream=stream)  # noqa: E731
        e2e_step()
        sync()
        e2e_steps = max(3, min(args.steps, 20))
        per_step = []

        def step_timer(fn, steps):       # the region on CUDA events, and each step's own time
            mean, region = time_launches(torch, fn, steps, stream, per_step)
            return region

        if sampler:
            sampler.pause()
        try:
            e2e_region = timed_replica_region(dist, e2e_step, e2e_steps, step_timer, sync)
        finally:
            if sampler:
                sampler.resume()
        e2e_ms, e2e_value, _ = replica_throughput(dist, e2e_region, e2e_steps, points, "cuda")

        def serial_step():   # for comparison: upload, kernel, download in sequence on one stream
            U.copy_(U_pin, non_blocking=True)
            binding.acs_rhs_saturated(U, R, stream=stream)
            R_pin.copy_(R, non_blocking=True)

        serial_step()
        sync()
        _, ser_region = time_launches(torch, serial_step, e2e_steps, stream)
        e2e = {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms, "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": out_bytes, "entry_point": "acs_rhs_saturated_host (pinned host U, R)",
               "step_ms_median": statistics.median(per_step), "step_ms_min": min(per_step),
               "step_ms_max": max(per_step),
               "clock_samples": "none: the NVML queries pause during this leg",
               "serial_copy_kernel_copy_ms": ser_region / e2e_steps,
               "host_link": host_link_floor(torch, U_pin, U, R, R_pin, stream, max(3, min(args.steps, 10)))}
        del ws_e2e

    # Star stencil, both forms, as context (one replica per rank, rank 0 reports).
    stencil = None
    if not args.no_stencil:
        del U, R
        torch.cuda.empty_cache()
        m = N_STAR
        u_np, a_np = inputs.stencil_fields(m, halo=4, seed=inputs.SEED_STENCIL)
        u = torch.from_numpy(u_np).to("cuda")
        a = torch.from_numpy(a_np).to("cuda")
        out = torch.empty((m, m, m), dtype=torch.float64, device="cuda")
        ssat = lambda: binding.acs_stencil_saturated(u, a, out, stream=stream)  # noqa: E731
        splain = lambda: binding.acs_stencil_plain(u, a, out, stream=stream)  # noqa: E731
        res = {}
        for name, fn in (("saturated", ssat), ("as_written", splain)):
            for _ in range(3):
                fn()
            sync()
            k = max(3, min(args.steps, 50))
            ta = time.time()
            lm, rm = time_launches(torch, fn, k, stream)
            if sampler:
                sampler.window(ta, time.time())
            res[name] = {"ms": rm / k, "gpts": m ** 3 / (rm / k * 1e-3) / 1e9}
        star_bytes = 8 * (2 * (m + 8) ** 3 + m ** 3)
        res["speedup"] = res["as_written"]["ms"] / res["saturated"]["ms"]
        star_gops = DP_OPS_PER_POINT["star_saturated"] * m ** 3 / (res["saturated"]["ms"] * 1e-3) / 1e9
        res["saturated"]["fp64_gops"] = star_gops
        res["saturated"]["fp64_frac"] = star_gops / probe["gops"]
        res["saturated"]["hbm_gbs_algorithmic"] = star_bytes / (res["saturated"]["ms"] * 1e-3) / 1e9
        stencil = {"grid": [m] * 3, "halo": 4, **res}
        del u, a, out
        torch.cuda.empty_cache()
        stencil["batch64"] = bench_batch(torch, binding, inputs, stream, max(3, min(args.steps, 50)))
        b = stencil["batch64"]["graph_autotuned"]
        b["fp64_frac"] = DP_OPS_PER_POINT["star_saturated"] * stencil["batch64"]["points"] / (b["ms"] * 1e-3) / 1e9 \
            / probe["gops"]

    if sampler:
        sampler.stop()
        clocks = sampler.summary()
        max_mhz = clocks.get("sm_max_mhz") or sampler.max_mhz
    else:
        clocks = None
        max_mhz = None
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    algo_bytes = in_bytes + out_bytes
    achieved_ops = DP_OPS_PER_POINT["rhs_saturated"] * points / (launch_ms * 1e-3) / 1e9
    derived = DP_OPS_PER_CLK_SM * sms * (max_mhz or FALLBACK_SM_MAX_MHZ) / 1000.0
    peak = probe["gops"]
    # the recorded figures are per 256^3 launch: other sizes report no traffic
    traffic = NCU_TRAFFIC.get(f"{kernel_source_hash()}:{tile_text(tuned_tile)}") if n == N_RHS else None
    result = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(n, world),
        "form": "saturated", "tile": tile_text(tuned_tile) + ("" if args.tile else " (acs_autotune_rhs)"),
        "roofline": {"bound": "alu", "achieved": achieved_ops, "peak": peak, "unit": "G FP64-pipe op/s",
                     "frac": achieved_ops / peak, "traffic": traffic,
                     "peak_source": "measured in this run: acs_fp64_rate_probe, register-only FP64 FMA chains at "
                                    f"{probe['blocks_per_sm']} blocks x {probe['threads']} threads per SM",
                     "peak_derived": derived,
                     "peak_derived_source": f"{DP_OPS_PER_CLK_SM} FP64 op/clk/SM x {sms} SMs (queried) x "
                                            f"{max_mhz or FALLBACK_SM_MAX_MHZ:.0f} MHz max SM clock "
                                            f"({'NVML' if max_mhz else 'fallback'})",
                     "frac_of_derived": achieved_ops / derived,
                     "sm_mhz_during_kernel": main_mhz},
        "fp64_probe": probe,
        "hbm": {"algorithmic_bytes_per_launch": algo_bytes, "achieved_gbs": algo_bytes / (launch_ms * 1e-3) / 1e9,
                "peak_gbs": hbm_peak, "frac": algo_bytes / (launch_ms * 1e-3) / 1e9 / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800"},
        "as_written": as_written,
        "ladder": ladder,
        "kernel_launch_ms": launch_ms,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "stencil_384": stencil,
    }
    if not args.no_stencil:
        result["block_128"] = bench_block(torch, binding, inputs, stream, max(3, min(args.steps, 20)))
    # The ranker study, the large workloads and the CPU baseline are single-GPU studies that rank 0
    # would run while the other ranks' GPUs stay held: the N = 1 line carries them.
    if world > 1:
        result["single_gpu_blocks"] = "ranker, large and cpu_baseline are reported at N = 1 only"
    if not args.no_ranker and world == 1:
        from paper_2306_13002_gb300 import ranker
        torch.cuda.empty_cache()
        study = bench_ranker(binding, ranker)
        keys = ("variants_generated", "variants_distinct", "train", "test", "fast_weight", "spearman_mlp_test",
                "spearman_analytical_test", "best_test_ms", "mlp_pick_ms", "analytical_pick_ms", "mlp_pick_over_best",
                "analytical_pick_over_best", "all_ms_min", "all_ms_median", "all_ms_max",
                "max_err_over_tol_vs_saturated", "mlp_pick_index", "mlp_pick_shape", "best_all_index",
                "mlp_top3_measured_over_best", "search", "splits",
                "wall_s")
        result["ranker"] = {"workload": f"march-scope rewriter variants of the RHS at {N_RHS}^3",
                            **{k: study[k] for k in keys},
                            "builtin_saturated_ms": ms_per_step,
                            "mlp_pick_over_builtin": study["mlp_pick_ms"] / ms_per_step}
        if not args.no_large:
            result["large"] = bench_large(torch, binding, inputs, stream, peak, study["mlp_pick_index"],
                                          max(3, min(args.steps, 10)))
    if not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(U_host)
    print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
