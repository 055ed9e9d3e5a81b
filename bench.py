#!/usr/bin/env python3
"""Benchmark of the fused RK4+2SHOC NLSE path on one GB300 (or N replicas).

Headline workload: 512 independent 2D NLSE instances of uneven size advanced
together -- sides U{64..1024 step 64} (seeded), a ~ U[0.3, 1], s = +-1,
V = w^2 r^2 with w ~ U[0, 0.1], Psi0 a Gaussian of width U[2, 8] with a
random phase gradient, Dirichlet boundaries, per-instance dt = 0.5 x the bound
of Eq. (kdfull) on Psi0.  One benchmark step is one full RK4 step of every
instance (four fused stage launches per tile group); the timed call is
nlse_run(K steps) with its device-side entry check, on the FP32 state with its
compensated part (FP64 invariants).  The default K = 5000 is the workload's
full length.

Reported beside it: the same batch in FP64 and the FP32-vs-FP64 error per
instance; the batch end to end through host buffers; the unfused FP64
schedule per instance; the 2D dark vortex on one 2048 x 2048 grid (FP32, FP64,
the multi-storage form, the unfused schedule, two stages per launch); the
gradient workload; the 3D vortex ring and the 1D soliton; and the CPU oracle,
all host cores and one, on a bounded sample of the batch.

``--impl reference`` times the CPU oracle instead (there is no other
implementation of the method to run), on all host cores, on a sample of the
batch sized so that the run ends in a few minutes.
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1109_1027_gb300 import workloads as wl  # noqa: E402

METRIC = "RK4 grid-pt updates/s & HBM GB/s vs ~8TB/s: FP32 batched vs FP64, at stated L2 err"
UNIT = "grid-point updates/s"
BATCH_COUNT = 512
BATCH_WORKLOAD = ("512 uneven 2D NLSE instances advanced together: sides U{64..1024 step 64} (seed 4), "
                  "a~U[0.3,1], s=+-1, V=w^2 r^2 with w~U[0,0.1], Gaussian psi0 of width U[2,8] with a phase "
                  "gradient, Dirichlet, per-instance dt = 0.5 dt_max(psi0) of Eq. (kdfull)")
N_SIDE = 2048
GRID_WORKLOAD = ("2D NLSE/GPE dark vortex 2048x2048 on [-60,60]^2, a=0.5, s=-1, V=0.01 r^2, "
                 "TF*tanh(r)*exp(i theta) + 1e-3 noise (seed 2), Dirichlet, dt = 0.5 dt_max")
# Algorithmic bytes per grid-point update of the FP32 compensated path: per
# RK4 step the four stages read/write (complex64 = 8 B, V float = 4 B)
#   stage 1: R Psi, V; W acc, Y                         = 28
#   stage 2: R Y, V, Psi, acc; W acc, Y                 = 44
#   stage 3: same                                       = 44
#   stage 4: R Y, V, Psi, lo, acc; W Psi, lo            = 52
BYTES_PER_UPDATE_FP32 = 168
# Two stages per launch (temporal blocking): stages 1+2 read Psi^n and V and
# write acc and Y_2 (28 B); stages 3+4 read Y_2, V, Psi^n, acc, lo and write
# Psi^{n+1} and lo (52 B).
BYTES_PER_UPDATE_FP32_FUSED = 80
# FP64 fused path (complex128 = 16 B, V double = 8 B, no low part): 56 + 88 + 88 + 72.
BYTES_PER_UPDATE_FP64 = 304
# The unfused FP64 schedule (complex128 16 B, V 8 B): 4 slopes x (D: R Y, W D = 32;
# step 2 + F: R Y, D, V, W K = 56) + 3 stage inputs (R Psi, K, W Y = 48) + the
# first increment (R K, W acc = 32) + 3 increments (R acc, K, W acc = 48) + the
# state update (R Psi, acc, W Psi = 48) = 352 + 144 + 32 + 144 + 48.
BYTES_PER_UPDATE_PLAIN = 720
# DRAM bytes per stage launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, the mean over the stage launches of consecutive RK4
# steps, with the L2 state of back-to-back steps: --cache-control none) for the
# kernel sources with the given hash; a kernel changed since its capture gets
# null.  Grid: 2048^2 dark vortex, mean of 12 launches.  Batch: the 512-instance
# batch with the default tile groups, mean of the wide-tile group's 8 launches
# (two steps), which covered `points` of the batch's points; the bench scales
# it to its own launches by points (the traffic is proportional to them).
NCU_TRAFFIC_GRID = {"93cfabc02338": 114148864}
NCU_TRAFFIC_BATCH = {"d8632e21fd29": {"bytes": 8571187616, "points": 198578176}}
# FP64 work per grid-point update (one RK4 step) of the FP64 stage kernels,
# from ncu instruction counts summed over the four stage launches of a step
# and divided by the points: flops = 2 x DFMA + DADD + DMUL, and instructions
# = DFMA + DADD + DMUL (each takes one FP64 issue slot).  Keyed by the source
# hash like the traffic.  2D: 2048^2 dark vortex; 3D: 256^3 vortex ring.
FP64_WORK_GRID = {"93cfabc02338": {"flops": 202.89, "instructions": 141.91}}
FP64_WORK_3D = {"05d6af1dabeb": {"flops": 264.27, "instructions": 203.26}}
# The gradient (FP32 state, FP64 dL/dV): per point and RK4 step the forward
# pass (168 B), the segment recompute (168 B: the same four stages, the stage
# inputs kept) and the four reversed stages.  Each reads its cotangent w (8),
# the stage input Y (8) and V (4) and writes lam (8); stages 4..2 write the
# next cotangent (8) and their dL/dV contribution (4); stages 3 and 2 read
# lam' (8; stage 4's w is lam' itself) and stages 3..1 the running lam (8);
# stage 1 reads the three contributions (12) and dL/dV (8, FP64) and writes
# dL/dV (8): 40 + 56 + 56 + 64 = 216 B.  Checkpoints (state and compensated
# part every 100 steps) add 0.6 B.
BYTES_PER_UPDATE_GRADIENT = 168 + 168 + 216
# Instances of the batch that the CPU oracle times (every 32nd).
CPU_SAMPLE_STRIDE = 32


def _hash(files) -> str:
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1109_1027_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_hash() -> str:
    """The single-grid 2D stage kernel's sources."""
    return _hash(("stage2d_tma.cuh", "stage2d_tile.cuh", "tma.cuh", "nlse_device.cuh"))


def batch_kernel_hash() -> str:
    """The batched 2D stage kernel's sources."""
    return _hash(("batch2d.cu", "stage2d_tile.cuh", "tma.cuh", "nlse_device.cuh"))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 50 ms, from before the
    autotuning of the headline leg to the end of its timed region; the
    summary takes the samples inside the marked timed window when there are
    at least three of them, else every sample of the leg (the same kernels
    under the same load)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS), "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def mark(self, t0: _dt.datetime, t1: _dt.datetime):
        """The timed region (local wall-clock times, as nvidia-smi prints them)."""
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    @staticmethod
    def _parse(ln):
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            return None
        try:
            ts = _dt.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            sm, mx = float(f[2]), float(f[3])
        except ValueError:
            return None
        return ts, sm, mx, f[6:10]

    def summary(self):
        rows = [r for r in (self._parse(ln) for ln in self.lines) if r is not None]
        where = "headline leg (tuning, warm-up, timed region)"
        if self.window is not None:
            pad = _dt.timedelta(milliseconds=self.PERIOD_MS)
            inside = [r for r in rows if self.window[0] - pad <= r[0] <= self.window[1] + pad]
            if len(inside) >= 3:
                rows, where = inside, "timed region"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "window": None}
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "window": where}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_barrier(pg, cuda: bool):
    """All ranks reach this point (and, on a GPU, have finished their work)."""
    if pg is not None:
        pg.barrier()
    if cuda:
        import torch
        torch.cuda.synchronize()


def ranks_max(pg, x: float, device="cpu") -> float:
    """The maximum of x over all ranks (x itself on one rank)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


def steps_taken(solver):
    """Raises if nlse_run's entry check refused the steps just timed (they did
    not run); a NaN or Inf produced by the steps themselves -- a collapsing
    focusing instance of the batch -- is reported elsewhere and does not void
    the timing."""
    from paper_1109_1027_gb300 import nlse
    try:
        solver.check()
    except nlse.NLSEError as err:
        if err.code == nlse.EUNSTABLE or "entry check" in str(err):
            raise


# -- CPU oracle (the cpu_baseline leg and the reference arm) -------------------

def batch_sample(insts, stride=CPU_SAMPLE_STRIDE):
    """Every stride-th instance of the batch: the sample the oracle times."""
    return [insts[i] for i in range(0, len(insts), stride)]


def oracle_batch_rate(sample, steps: int | None, seconds: float, threads: int):
    """Times the FP64 CPU oracle on the sampled instances: each benchmark step
    is one RK4 step of every sampled instance.  With steps None, as many steps
    as fit in about `seconds`."""
    import oracle
    probs, states, Vs, ks = [], [], [], []
    for q in sample:
        prob = oracle.Problem(q.shape, q.h, q.a, q.s)
        probs.append(prob)
        states.append(q.psi0.copy())
        Vs.append(q.V)
        ks.append(0.5 * oracle.invariants(prob, q.psi0, q.V)[2])
    pts = sum(int(np.prod(q.shape)) for q in sample)

    def step_all():
        for i in range(len(sample)):
            states[i] = oracle.run(probs[i], states[i], Vs[i], ks[i], 1, threads=threads)

    if steps is None:
        t0 = time.perf_counter()
        step_all()
        per = time.perf_counter() - t0
        steps = max(2, int(seconds / per))
    t0 = time.perf_counter()
    for _ in range(steps):
        step_all()
    el = time.perf_counter() - t0
    return pts * steps / el, pts, steps, el


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    threads = oracle.threads_available()
    used = oracle.threads_used(threads)
    insts = wl.gaussian_batch_2d(count=BATCH_COUNT, seed=4, steps=0,
                                 only=set(range(0, BATCH_COUNT, CPU_SAMPLE_STRIDE)))
    sample = sorted(insts, key=lambda q: q.shape[0])
    # keep the smallest sampled instances that fit ~120 s for warmup + steps
    probe = sample[: max(1, len(sample) // 2)]
    _, ppts, _, pel = oracle_batch_rate(probe, 1, 0, threads)
    per_point = pel / ppts
    budget = 120.0 / max(1, args.steps + args.warmup)
    chosen, pts = [], 0
    for q in sample:
        n = int(np.prod(q.shape))
        if chosen and (pts + n) * per_point > budget:
            break
        chosen.append(q)
        pts += n
    oracle_batch_rate(chosen, args.warmup, 0, threads)              # warm-up steps
    value, pts, _, el = oracle_batch_rate(chosen, args.steps, 0, threads)
    sample_txt = (f"{len(chosen)} instances of the batch (every {CPU_SAMPLE_STRIDE}th, smallest first; "
                  f"{pts} points, sides {[q.shape[0] for q in chosen]}), one RK4 step of each per benchmark step, "
                  f"FP64 C oracle on {used} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": BATCH_WORKLOAD, "sample": sample_txt},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample_txt},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# -- the GPU arm -----------------------------------------------------------------

def timed(fn, stream, barrier, max_over_ranks):
    """Milliseconds of fn() on the stream (CUDA events), max over ranks."""
    import torch
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1))


def run_ours(args):
    import torch

    from paper_1109_1027_gb300 import autotune, nlse

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    nlse.load_library()
    stream = torch.cuda.current_stream()
    barrier = lambda: rank_barrier(pg, cuda=True)
    max_over_ranks = lambda x: ranks_max(pg, x, dev)
    K, W = args.steps, args.warmup

    # ---- the batch: independent instances, one differently seeded batch per rank ----
    insts = wl.gaussian_batch_2d(count=BATCH_COUNT, seed=4 + rank, steps=0)
    shapes = [q.shape for q in insts]
    npts = sum(q.shape[0] * q.shape[1] for q in insts)
    hs, as_, ss = [q.h for q in insts], [q.a for q in insts], [q.s for q in insts]
    V64 = nlse.BatchSolver.pack([q.V for q in insts], torch.float64, dev)
    psi64 = nlse.BatchSolver.pack([q.psi0 for q in insts], torch.complex128, dev)
    probe = nlse.BatchSolver(V64, shapes, hs, 1.0, as_, ss, prec="fp64", check_stability=False)
    _, _, dtmax = probe.invariants(psi64)
    probe.close()
    dts = [0.5 * d for d in dtmax]
    V32 = V64.float().contiguous()
    psi32 = psi64.to(torch.complex64).contiguous()

    # ---- headline: the batch in FP32, nlse_run(K) with its entry check ------------
    b32 = nlse.BatchSolver(V32, shapes, hs, dts, as_, ss, prec="fp32")
    x32 = psi32.clone()
    with ClockSampler(local) as clk:
        tuning = autotune.tune(b32, x32, steps=3, use_cache=False)
        b32.run(x32, W)
        steps_taken(b32)
        t_start = _dt.datetime.now()
        ms = timed(lambda: b32.run(x32, K), stream, barrier, max_over_ranks)
        t_end = _dt.datetime.now()
        clk.mark(t_start, t_end)
    steps_taken(b32)
    clocks = clk.summary()
    narrow = b32.get_tiling(nlse.TILE_BATCH_NARROW)
    groups = int(any(sh[1] <= narrow for sh in shapes)) + int(any(sh[1] > narrow for sh in shapes))
    ms_step = ms / K
    value = job_rate(world, npts * K, ms * 1e-3)
    launches = 4 * groups * K + 2

    # ---- this GPU's FP64 rate, the denominator of the FP64 legs' roofline ----------
    fp64_peak = nlse.nlse_measure_fp64_rate()

    # ---- the same batch in FP64 ----------------------------------------------------
    k64 = min(K, 50)
    b64 = nlse.BatchSolver(V64, shapes, hs, dts, as_, ss, prec="fp64")
    x64 = psi64.clone()
    b64.run(x64, 3)
    steps_taken(b64)
    ms64 = timed(lambda: b64.run(x64, k64), stream, barrier, max_over_ranks)
    steps_taken(b64)

    # ---- FP32 vs FP64 after the error run (per instance, relative L2) ---------------
    ke = args.batch_steps
    x32.copy_(psi32)
    b32.reset_compensation()
    x64.copy_(psi64)
    b32.run(x32, ke)
    b64.run(x64, ke)
    for sv in (b32, b64):
        try:
            sv.check()
        except nlse.NLSEError as err:
            if err.code != nlse.ENONFINITE or "entry check" in str(err):
                raise
    errs, collapsed = {-1: [], 1: []}, 0
    a64, a32 = x64, x32.to(torch.complex128)
    off = 0
    for q in insts:
        n = q.shape[0] * q.shape[1]
        s64, s32 = a64[off:off + n], a32[off:off + n]
        off += n
        if not (bool(torch.isfinite(s64).all()) and bool(torch.isfinite(s32).all())):
            collapsed += 1
            continue
        errs[1 if q.s > 0 else -1].append(float(torch.linalg.vector_norm(s32 - s64) / torch.linalg.vector_norm(s64)))
    del a32

    def stats(e):
        e = sorted(e)
        return {"max": e[-1], "median": e[len(e) // 2], "instances": len(e),
                "within_1e-5": sum(v <= 1e-5 for v in e)} if e else None

    # ---- end to end: the batch state in pinned host memory ------------------------
    kh_e2e = min(K, 20)
    host = psi32.cpu().pin_memory()
    be = nlse.BatchSolver(V32, shapes, hs, dts, as_, ss, prec="fp32", check_stability=False)
    be.set_tiling(nlse.TILE_BATCH_NARROW, narrow)

    def host_steps(n):
        for _ in range(n):
            try:
                be.run_host(host, 1)
            except nlse.NLSEError as err:     # a focusing instance collapsing; reported above
                if err.code != nlse.ENONFINITE:
                    raise

    host_steps(3)
    mse = timed(lambda: host_steps(kh_e2e), stream, barrier, max_over_ranks)
    be.close()
    e2e_value = job_rate(world, npts * kh_e2e, mse * 1e-3)
    cbytes = npts * 8
    del host

    # ---- roofline of the batched stage kernel --------------------------------------
    peak, peak_kind = load_peaks()
    achieved = BYTES_PER_UPDATE_FP32 * npts / (ms_step * 1e-3) / 1e9
    bkh = batch_kernel_hash()
    cap = NCU_TRAFFIC_BATCH.get(bkh)
    traffic = cap["bytes"] * npts / cap["points"] if cap else None      # per stage pass over the whole batch
    launch_ms = ms_step / 4
    roofline = {"bound": "hbm", "kernel": "stage2d_batch_kernel<float> (RK4 stages 1-4 over the batch, mean per "
                                          "stage; both tile groups of a stage counted as one pass)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": BYTES_PER_UPDATE_FP32 / 4 * npts,
                "launch_ms": launch_ms,
                "traffic": traffic,
                "traffic_what": "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean per stage launch of the "
                                "wide-tile group, scaled to all of the batch's points",
                "dram_gbs": traffic / (launch_ms * 1e-3) / 1e9 if traffic else None,
                "dram_frac": traffic / (launch_ms * 1e-3) / 1e9 / peak if traffic else None,
                "kernel_hash": bkh}

    # ---- the unfused FP64 schedule, one context per instance --------------
    plain = None
    if not args.quick:
        sample = list(range(0, len(insts), 8))
        pst = 10
        offs = np.cumsum([0] + [q.shape[0] * q.shape[1] for q in insts])
        solvers, states = [], []
        for i in sample:
            q = insts[i]
            Vi = V64[offs[i]:offs[i + 1]].reshape(q.shape).contiguous()
            solvers.append(nlse.Solver(Vi, q.h, dts[i], q.a, q.s, prec="fp64", plain=True, check_stability=False))
            states.append(psi64[offs[i]:offs[i + 1]].reshape(q.shape).contiguous().clone())
        for sv, xs in zip(solvers, states):
            sv.run(xs, 2)

        def plain_steps():
            for sv, xs in zip(solvers, states):
                sv.run(xs, pst)

        msp = timed(plain_steps, stream, barrier, max_over_ranks)
        spts = sum(insts[i].shape[0] * insts[i].shape[1] for i in sample)
        for sv in solvers:
            sv.close()
        plain = {"value": job_rate(world, spts * pst, msp * 1e-3), "unit": UNIT, "instances": len(sample),
                 "points": int(spts), "steps": pst,
                 "what": "unfused FP64 schedule, one context per instance, instances in sequence "
                         "(every 8th instance of the batch)"}
    b32.close()
    b64.close()
    del x32, x64, psi64, V64

    grid = None if args.quick else run_grid_legs(args, dev, rank, world, stream, barrier, max_over_ranks, fp64_peak)
    grad = None if args.quick else run_gradient_leg(args, dev, barrier, max_over_ranks)
    other = None if args.quick else run_other_grids(dev, barrier, max_over_ranks, fp64_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        sample = batch_sample(insts)
        threads = oracle.threads_available()
        used = oracle.threads_used(threads)
        rate_all, spts, st_all, sec_all = oracle_batch_rate(sample, None, 12.0, threads)
        rate_one, _, st_one, sec_one = oracle_batch_rate(sample, None, 8.0, 1)
        what = (f"FP64 C oracle on every {CPU_SAMPLE_STRIDE}th instance of the batch ({len(sample)} instances, "
                f"{spts} points), one RK4 step of each per step")
        cpu = {"value": rate_all, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"{what}; {st_all} steps in {sec_all:.1f} s on {used} threads",
               "single_thread": {"value": rate_one, "unit": UNIT, "cores": 1,
                                 "sample": f"{what}; {st_one} steps in {sec_one:.1f} s"}}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances": BATCH_COUNT, "points": npts,
                       "precision": "complex64 state + compensated low part, FP64 invariants and entry check",
                       "l2_cache": f"working set {npts * 44 / 2**30:.1f} GiB (Psi, lo, 2 stage buffers, acc, V) "
                                   "> 126 MiB L2; no flush",
                       "parallelism": f"{world} independent batch(es), one per rank",
                       "tiling": {"narrow_tile_width_bound": narrow, "chosen_by": "autotune (timed on this batch)",
                                  "ms_per_step": {str(k_): v["ms_per_step"] for k_, v in tuning.items()}}},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": cbytes, "d2h_bytes_per_step": cbytes,
                    "steps": kh_e2e,
                    "what": "per step: nlse_run_host(1 step) on the batch state in pinned host memory: H2D of "
                            "Psi, one RK4 step, D2H of Psi and the status, stream synchronised (entry check "
                            "off: the workload's focusing instances collapse and fall below their bound)"},
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_peak": {"value": fp64_peak / 1e12, "unit": "TFLOP/s",
                          "how": "nlse_measure_fp64_rate: 8 independent FMA chains per thread, 8 CTAs of 256 "
                                 "threads per SM, best of three launches (CUDA events)"},
            "batched_fp64": {"value": job_rate(world, npts * k64, ms64 * 1e-3), "unit": UNIT, "steps": k64,
                             "ms_per_step": ms64 / k64,
                             "achieved_gbs": BYTES_PER_UPDATE_FP64 * npts / (ms64 / k64 * 1e-3) / 1e9},
            "batched_fp32_vs_fp64_rel_l2": {"steps": ke, "defocusing_s-1": stats(errs[-1]),
                                            "focusing_s+1": stats(errs[1]), "collapsed_instances": collapsed,
                                            "collapsed_note": "focusing (s=+1) instances whose mass exceeds the "
                                            "2D critical mass collapse; with dt fixed at 0.5 dt_max(psi0) the "
                                            "explicit scheme then overflows (the bound of Eq. kdfull shrinks as "
                                            "|psi| grows); they are excluded from the error statistics"},
            "batched_fp64_plain_per_instance": plain,
            "grid_2048": grid,
            "gradient": grad,
            "other_grids": other,
        }))
    if pg is not None:
        pg.destroy_process_group()


def run_grid_legs(args, dev, rank, world, stream, barrier, max_over_ranks, fp64_peak):
    """The 2D dark vortex on one 2048 x 2048 grid: FP32 (autotuned), the other
    FP32 launch schedule, FP64 fused, FP64 multi-storage, the unfused
    FP64 schedule; FP32-vs-FP64 difference, mass and energy drift."""
    import torch

    from paper_1109_1027_gb300 import autotune, nlse

    K, W = min(args.steps, 2000), args.warmup
    inst = wl.dark_vortex_2d(n=N_SIDE, seed=2 + rank, steps=0)
    npts = N_SIDE * N_SIDE
    V32 = torch.from_numpy(inst.V).to(dev).float().contiguous()
    V64 = torch.from_numpy(inst.V).to(dev).contiguous()
    psi0 = torch.from_numpy(inst.psi0).to(dev)
    probe = nlse.Solver(V64, inst.h, 1.0, inst.a, inst.s, prec="fp64", check_stability=False)
    _, _, dtmax = probe.invariants(psi0.clone())
    probe.close()
    k = 0.5 * dtmax
    out = {"workload": GRID_WORKLOAD, "steps": K, "dt": k}

    s32 = nlse.Solver(V32, inst.h, k, inst.a, inst.s, prec="fp32")
    x32 = psi0.to(torch.complex64).contiguous()
    tuning = autotune.tune(s32, x32, use_cache=False)
    s32.run(x32, W)
    ms = timed(lambda: s32.run(x32, K), stream, barrier, max_over_ranks)
    steps_taken(s32)
    rows, fused = s32.get_tiling(nlse.TILE_ROWS), s32.get_tiling(nlse.TILE_2D_FUSE)
    ms_step = ms / K
    peak, peak_kind = load_peaks()
    bpu = BYTES_PER_UPDATE_FP32_FUSED if fused else BYTES_PER_UPDATE_FP32
    nl = 2 if fused else 4
    kh = kernel_hash()
    traffic = None if fused else NCU_TRAFFIC_GRID.get(kh)
    achieved = bpu * npts / (ms_step * 1e-3) / 1e9
    out["fp32"] = {"value": job_rate(world, npts * K, ms * 1e-3), "unit": UNIT, "ms_per_step": ms_step,
                   "tiling": {"rows_per_cta": rows, "two_stages_per_launch": fused,
                              "ms_per_step": {str(k_): v["ms_per_step"] for k_, v in tuning.items()}},
                   "roofline": {"bound": "hbm", "kernel": "rk4_2d_fused_kernel" if fused else "stage2d_tma_kernel<float>",
                                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                "peak_kind": f"{peak_kind} copy bandwidth",
                                "algorithmic_bytes_per_launch": bpu / nl * npts, "launch_ms": ms_step / nl,
                                "traffic": traffic,
                                "dram_gbs": traffic / (ms_step / nl * 1e-3) / 1e9 if traffic else None,
                                "kernel_hash": kh}}

    # the launch schedule the autotuner did not keep (same bits)
    kf = min(K, 1000)
    sf = nlse.Solver(V32, inst.h, k, inst.a, inst.s, prec="fp32")
    sf.set_tiling(nlse.TILE_ROWS, rows)
    sf.set_tiling(nlse.TILE_2D_FUSE, 1 - fused)
    xa = psi0.to(torch.complex64).contiguous()
    xb = psi0.to(torch.complex64).contiguous()
    s32.run(xa, 64)
    sf.run(xb, 64)
    same_bits = bool(torch.equal(xa, xb))
    sf.run(xb, W)
    msf = timed(lambda: sf.run(xb, kf), stream, barrier, max_over_ranks)
    steps_taken(sf)
    sf.close()
    del xa, xb
    bpu_f = BYTES_PER_UPDATE_FP32 if fused else BYTES_PER_UPDATE_FP32_FUSED
    out["fp32_other_schedule"] = {
        "schedule": "four single-stage launches per step" if fused else
                    "two launches per step, two RK4 stages each (temporal blocking)",
        "value": job_rate(world, npts * kf, msf * 1e-3), "unit": UNIT, "steps": kf, "ms_per_step": msf / kf,
        "bytes_per_update": bpu_f, "achieved_gbs": bpu_f * npts / (msf / kf * 1e-3) / 1e9,
        "same_bits_as_the_kept_schedule_after_64_steps": same_bits}

    x32.copy_(psi0.to(torch.complex64))
    s32.reset_compensation()
    s64 = nlse.Solver(V64, inst.h, k, inst.a, inst.s, prec="fp64")
    x64 = psi0.clone().contiguous()
    s64.run(x64, W)
    x64.copy_(psi0)
    ms64 = timed(lambda: s64.run(x64, K), stream, barrier, max_over_ranks)
    steps_taken(s64)
    s32.run(x32, K)
    steps_taken(s32)
    rate64 = npts * K / (ms64 * 1e-3)
    out["fp64"] = {"value": job_rate(world, npts * K, ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / K,
                   "achieved_gbs": BYTES_PER_UPDATE_FP64 * npts / (ms64 / K * 1e-3) / 1e9,
                   "roofline": fp64_roofline(FP64_WORK_GRID.get(kh), rate64, fp64_peak, "stage2d_tma_kernel<double>",
                                             kh)}
    out["fp32_vs_fp64_rel_l2_after_steps"] = float(
        torch.linalg.vector_norm(x32.to(torch.complex128) - x64) / torch.linalg.vector_norm(x64))
    m32, en32, _ = s32.invariants(x32)
    m64, en64, _ = s64.invariants(x64)
    m0, en0, _ = s64.invariants(psi0.clone())
    out["mass_drift"] = {"fp32": m32 / m0 - 1, "fp64": m64 / m0 - 1}
    out["energy_drift"] = {"fp32": en32 / en0 - 1, "fp64": en64 / en0 - 1}

    # the cost of a look at the invariants (FP64 reductions, one synchronising call each)
    def inv_ms(solver, x, energy):
        solver.invariants(x, energy=energy)
        t0 = time.perf_counter()
        for _ in range(5):
            solver.invariants(x, energy=energy)
        return (time.perf_counter() - t0) / 5 * 1e3
    out["invariants_ms_per_call"] = {"fp32": inv_ms(s32, x32, True), "fp32_without_energy": inv_ms(s32, x32, False),
                                     "fp64": inv_ms(s64, x64, True),
                                     "what": "nlse_invariants on the grid (mass, energy, dt_max; host clock "
                                             "around the synchronising call)"}

    # FP64 with the multi-storage 2SHOC form (Eqs. 2d2shocMs1-2)
    kms = min(K, 500)
    sm = nlse.Solver(V64, inst.h, k, inst.a, inst.s, prec="fp64", lap="2shoc_ms")
    xm = psi0.clone().contiguous()
    sm.run(xm, W)
    xm.copy_(psi0)
    msm = timed(lambda: sm.run(xm, kms), stream, barrier, max_over_ranks)
    steps_taken(sm)
    sm.close()
    xs = psi0.clone().contiguous()
    s64.run(xs, kms)
    out["fp64_multi_storage"] = {"value": job_rate(world, npts * kms, msm * 1e-3), "unit": UNIT, "steps": kms,
                                 "ms_per_step": msm / kms,
                                 "rel_l2_vs_single_storage": float(torch.linalg.vector_norm(xm - xs) /
                                                                   torch.linalg.vector_norm(xs))}
    del xs, xm

    # the unfused FP64 schedule on the same GPU (baseline)
    kp = min(K, 500)
    sp = nlse.Solver(V64, inst.h, k, inst.a, inst.s, prec="fp64", plain=True)
    xp = psi0.clone().contiguous()
    sp.run(xp, W)
    msp = timed(lambda: sp.run(xp, kp), stream, barrier, max_over_ranks)
    steps_taken(sp)
    sp.close()
    out["fp64_plain"] = {"value": job_rate(world, npts * kp, msp * 1e-3), "unit": UNIT, "steps": kp,
                         "ms_per_step": msp / kp,
                         "achieved_gbs": BYTES_PER_UPDATE_PLAIN * npts / (msp / kp * 1e-3) / 1e9,
                         "what": "unfused schedule: D and the RK4 work fields in HBM, 16 launches per step"}
    s32.close()
    s64.close()
    return out


def fp64_roofline(work, rate, fp64_peak, kernel, kh):
    """ALU roofline of an FP64 stage kernel: achieved FP64 flops against the
    measured FMA rate, and the FP64 issue slots used (one per DFMA, DADD or
    DMUL) against the slots that rate implies (half the flop rate)."""
    out = {"bound": "alu", "kernel": kernel, "achieved": None, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
           "frac": None, "peak_kind": "measured FP64 FMA rate (nlse_measure_fp64_rate)", "kernel_hash": kh}
    if work:
        out.update(achieved=work["flops"] * rate / 1e12, frac=work["flops"] * rate / fp64_peak,
                   flops_per_update=work["flops"], fp64_instructions_per_update=work["instructions"],
                   fp64_issue_frac=work["instructions"] * rate / (fp64_peak / 2))
    return out


def run_other_grids(dev, barrier, max_over_ranks, fp64_peak):
    """Step rates of the 3D vortex ring (512^3) and the 1D bright soliton
    (2048 points, the whole 2000-step run) in FP32 and FP64."""
    import torch

    from paper_1109_1027_gb300 import autotune, nlse

    out = {}
    stream = torch.cuda.current_stream()

    def rate(inst, prec, steps, lap="2shoc"):
        rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
        V = torch.from_numpy(inst.V).to(dev).to(rdt).contiguous()
        x = torch.from_numpy(inst.psi0).to(dev).to(cdt).contiguous()
        probe = nlse.Solver(V, inst.h, 1.0, inst.a, inst.s, prec=prec, check_stability=False)
        dtm = probe.invariants(x)[2]
        probe.close()
        sv = nlse.Solver(V, inst.h, 0.5 * dtm, inst.a, inst.s, prec=prec, lap=lap)
        autotune.tune(sv, x, steps=4, use_cache=False)
        sv.run(x, 3)
        ms = timed(lambda: sv.run(x, steps), stream, barrier, max_over_ranks) / steps
        steps_taken(sv)
        npts = int(np.prod(inst.shape))
        res = {"ms_per_step": ms, "updates_per_s": npts / (ms * 1e-3)}
        if len(inst.shape) == 1 and sv.get_tiling(nlse.TILE_1D_RESIDENT):
            # The whole run is one launch with the state on chip: no HBM traffic per step.
            res["path"] = f"one launch for all {steps} steps, cluster of up to {sv.get_tiling(nlse.TILE_1D_RESIDENT)} CTAs"
        else:
            bpu = BYTES_PER_UPDATE_FP32 if prec == "fp32" else BYTES_PER_UPDATE_FP64
            res["achieved_gbs"] = bpu * npts / (ms * 1e-3) / 1e9
        if len(inst.shape) == 3 and prec == "fp64" and lap == "2shoc":
            kh3 = _hash(("stage3d.cu", "nlse_device.cuh"))
            res["roofline"] = fp64_roofline(FP64_WORK_3D.get(kh3), npts / (ms * 1e-3), fp64_peak,
                                            "stage3d_kernel<double>", kh3)
        sv.close()
        return res

    ring = wl.vortex_ring_3d(n=512, steps=0)
    out["vortex_ring_3d_512"] = {"fp32": rate(ring, "fp32", 40), "fp64": rate(ring, "fp64", 8),
                                 "fp32_multi_storage": rate(ring, "fp32", 40, "2shoc_ms")}
    del ring
    sol = wl.bright_soliton_1d()
    out["bright_soliton_1d_2048"] = {"fp32": rate(sol, "fp32", 2000), "fp64": rate(sol, "fp64", 2000)}
    return out


def run_gradient_leg(args, dev, barrier, max_over_ranks):
    """dL/dpsi0 and dL/dV of L = sum |Psi_T - target|^2 for the gradient
    workload: 16 initial states on a 512 x 512 grid, a = 0.5, s = -1,
    V = harmonic + seeded 8x8 Fourier-mode perturbation, complex64 state with
    FP64 loss and dL/dV accumulation, checkpoints every 100 steps."""
    import torch

    from paper_1109_1027_gb300 import nlse

    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=512, batch=16)
    Vd = torch.from_numpy(V).to(dev).float().contiguous()
    probe = nlse.Solver(torch.from_numpy(V).to(dev), h, 1.0, a, s, prec="fp64", check_stability=False)
    dt = 0.5 * min(probe.invariants(torch.from_numpy(p).to(dev).contiguous())[2] for p in psis)
    probe.close()
    steps = args.grad_steps
    # The 16 initial states share V: one stacked context advances them in one
    # launch per stage (NLSE_FLAG_STACK) and returns the summed loss and dL/dV.
    x0 = torch.stack([torch.from_numpy(p).to(torch.complex64) for p in psis]).to(dev).contiguous()
    tg = torch.stack([torch.from_numpy(t).to(torch.complex64) for t in targets]).to(dev).contiguous()
    sv = nlse.Solver(Vd, h, dt, a, s, prec="fp32", check_stability=False, stack=len(psis))
    sv.adjoint(x0, tg, 10, 5)                                      # warm-up
    barrier()
    t0 = time.perf_counter()
    loss, _, gV = sv.adjoint(x0, tg, steps, 100)
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0)
    sv.close()
    return {"workload": "16 x 512^2, a=0.5, s=-1, V = 0.01 r^2 + 8x8 Fourier modes (seed 5), Gaussian psi0/targets",
            "steps": steps, "checkpoint_every": 100, "batch": 16, "seconds_per_batch_gradient": el,
            "how": "one stacked context (NLSE_FLAG_STACK): the 16 instances share V and advance in one launch "
                   "per stage; dL/dV summed over the instances in FP64",
            "forward_equivalent_updates_per_s": 16 * 512 * 512 * steps / el,
            "roofline": {"bound": "hbm", "kernel": "forward + recompute stages and adj2d_kernel, whole gradient",
                         "bytes_per_update": BYTES_PER_UPDATE_GRADIENT,
                         "achieved": BYTES_PER_UPDATE_GRADIENT * 16 * 512 * 512 * steps / el / 1e9,
                         "peak": load_peaks()[0], "unit": "GB/s",
                         "frac": BYTES_PER_UPDATE_GRADIENT * 16 * 512 * 512 * steps / el / 1e9 / load_peaks()[0]},
            "loss_sum": float(loss), "dV_norm": float(torch.linalg.vector_norm(gV))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="the batched headline, its FP64 and e2e legs only")
    ap.add_argument("--batch-steps", type=int, default=200, help="steps of the FP32-vs-FP64 error run")
    ap.add_argument("--grad-steps", type=int, default=3000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
