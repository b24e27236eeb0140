#!/usr/bin/env python3
"""Benchmark: pair-interactions/s of the level-0 GENGA step with the FP32
long-range kick on a 40,000-body disc, against the FP64 kick on the same GPU.

One step = kick(dt/2) + drift(dt) + kick(dt/2) through the C ABI
(genga_step), i.e. two long-range passes of N(N-1) pair interactions each,
plus the Eq. (1) radius, packing, encounter list and Kepler drift.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl genga|reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica disc (seed 3 + rank): the discs share nothing, so there
is no collective on the data path ("scaling": "weak"); the barrier and the
max over ranks are only for timing.

--impl reference times the CPU FP64 oracle on the host cores on bounded
samples of the same workload (rows of the pair sum) and prints the same line
with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s, FP32 vs FP64 kick, N=40k, 1 GB300, accel rel-err≤2e-5"
UNIT = "pair-interactions/s"
WORKLOAD = ("disc40k: 40,000 equal-mass planetesimals (5 Earth masses), surface density ~ a^-1.5 on "
            "0.5-4 au, e/i Rayleigh 0.01/0.005, dt = 6 d, r_crit = 3 mutual Hill radii, Chambers changeover")
FLOPS_PER_PAIR = 20          # the usual convention for one gravitational pair interaction
L2_FLUSH_BYTES = 512 << 20   # larger than the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="genga", choices=["genga", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variant", type=int, default=-1, help="force an FP32 pass variant (-1: autotune)")
    ap.add_argument("--fp64-variant", type=int, default=-1, help="force an FP64 pass variant (-1: autotune)")
    ap.add_argument("--no-sweep", action="store_true", help="skip timing every FP32 variant")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-disc batched workload")
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--no-tp2", action="store_true", help="skip the test-particle-mode-2 kicks on giants100k")
    ap.add_argument("--long-steps", type=int, default=1000,
                    help="length of the run whose mean step and pass times are reported (0: skip)")
    ap.add_argument("--no-levels", action="store_true", help="skip the intermediate-levels object")
    ap.add_argument("--levels", default=None,
                    help="L:s -- time the disc40k steps of the 'levels' object with L intermediate levels of s "
                         "sub-steps instead of the tuned setting")
    ap.add_argument("--bs-tol", type=float, default=1e-12,
                    help="tolerance of the close-encounter (Bulirsch-Stoer) level, timed beside the headline "
                         "step (which is the level-0 path: kick, drift, kick); 0: skip that measurement")
    ap.add_argument("--conservation", default=None,
                    help="instead of the benchmark: energy and angular-momentum drift of FP32 vs FP64 runs, "
                         "comma-separated workload:steps:sample_every[:n_big] (e.g. "
                         "embryo6625:100000:5000,giants100k:10000:500:4; n_big: test-particle mode 2)")
    return ap.parse_args()


# ------------------------------------------------------------- clocks -----
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        try:
            smax = float(rows[0][2])
        except ValueError:
            smax = None
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


# -------------------------------------------------------------- helpers ---
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank):
    """Seed of the disc a rank steps: rank 0 runs the disc40k workload itself
    (seed 3); every other rank an independent replica of the same recipe."""
    return 3 + rank


def max_over_ranks(x, dist=None, device=None):
    """The slowest rank's time (the job ends when the last rank does)."""
    if dist is None or not dist.is_initialized():
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(ws, pairs_per_step, steps, ms_max):
    """Whole-job pair-interactions/s: every rank did `steps` steps of its own
    replica, the job took the slowest rank's time."""
    return ws * pairs_per_step * steps / (ms_max * 1e-3)


KERNEL_SOURCE = {"pass_fp32_kernel": "kick.cu", "pass_mutual_kernel": "mutual.cu", "pass_fp64_kernel": "kick.cu",
                 "pass_mutual64_kernel": "mutual.cu"}


def kernel_traffic(kernel):
    """dram bytes per launch of a pass kernel from the committed ncu summary
    (profiles/traffic.json, one record per kernel), or None when there is no
    record or the kernel's source file has changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCE:
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2309_08217_gb300", "csrc", KERNEL_SOURCE[kernel])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("source_sha256") != sha:
        return None
    return rec.get("dram_bytes_per_launch")


def oracle_sample_rate(d, seconds, seed=0):
    """Time the FP64 oracle's pair sum on a bounded sample of body rows;
    returns (pairs/s, rows, threads, acc rows, row indices)."""
    import numpy as np

    import oracle
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    rng = np.random.default_rng(seed)
    # calibrate on a few rows, then size the sample to the time budget
    rows = 64
    idx = np.sort(rng.choice(d.N, rows, replace=False))
    t0 = time.perf_counter()
    oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx)
    dt_cal = time.perf_counter() - t0
    rows = int(min(d.N, max(64, rows * seconds / max(dt_cal, 1e-6))))
    idx = np.sort(rng.choice(d.N, rows, replace=False))
    t0 = time.perf_counter()
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx)
    el = time.perf_counter() - t0
    return rows * (d.N - 1) / el, rows, oracle.threads(), acc, idx, el


# ------------------------------------------------------------ reference ---
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2309_08217_gb300 import discs
    d = discs.workload("disc40k")
    budget = max(1.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(d, budget / 4)
    rates, rows_all, el_all, thr = [], 0, 0.0, 1
    for k in range(args.steps):
        rate, rows, thr, _, _, el = oracle_sample_rate(d, budget, seed=k + 1)
        rates.append(rate)
        rows_all += rows
        el_all += el
    value = rows_all * (d.N - 1) / el_all
    pairs_step = 2 * d.N * (d.N - 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": pairs_step / value * 1e3,
        "ms_per_step_how": "derived, not timed: pairs_per_step / value (the oracle is timed on row samples "
                           "of the pair sum, not on whole steps)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": d.N, "pairs_per_step": pairs_step,
                   "sample": "each step: the oracle's FP64 pair sum over a random sample of body rows "
                             f"({rows_all // max(1, args.steps)} rows x {d.N - 1} partners on average)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{rows_all} body rows over {args.steps} steps, {el_all:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- batched ----
BATCH_WORKLOAD = ("batch256: 256 independent discs, N_d = floor(exp U(ln 1000, ln 16000)) planetesimals each "
                  "(2.5 Earth masses, 0.5-4 au), FP32 kick, dt = 6 d")


def run_batched(g, torch, dev, stream, flush, args, rank, ws=1, dist=None):
    """genga_step_batched over 256 discs against genga_step on each disc in turn."""
    import numpy as np
    from paper_2309_08217_gb300 import discs
    ds = discs.batch_of_discs(256, 4 + 1000 * rank)
    sizes = np.array([d.N for d in ds])
    offsets = np.concatenate([[0], np.cumsum(sizes)]).tolist()
    padded = int(sum((n + 1023) // 1024 * 1024 for n in sizes))
    pairs_step = 2 * int((sizes * (sizes - 1)).sum())
    p = g.make_params(G=ds[0].G, Mstar=1.0, dt=6.0, precision=g.GENGA_FP32)
    K, W = max(1, args.batched_steps), 3

    def timed(step_once):
        for _ in range(W):
            step_once()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize(dev)
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            step_once()
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in evs)

    ctxb = g.Context(padded, dev.index)
    allsys = g.DeviceSystem.from_arrays([np.concatenate([d.arrays()[c] for d in ds]) for c in range(7)], device=dev)
    ms_b = timed(lambda: g.genga_step_batched(ctxb, allsys, offsets, p, 1))
    g.genga_step_batched(ctxb, allsys, offsets, p, 8)     # align the order, capture the 4-step graph
    ms_bg = timed(lambda: g.genga_step_batched(ctxb, allsys, offsets, p, 4)) / 4
    if g.genga_get_status(ctxb) != g.GENGA_OK:
        raise RuntimeError("device status after the batched steps")
    bvar, bms = g.genga_batched_tuning(ctxb, offsets)
    ctxb.close()
    ctxs = g.Context(int(sizes.max()), dev.index)
    systems = [g.DeviceSystem.from_disc(d, device=dev) for d in ds]

    def sequential():
        for sd in systems:
            g.genga_step(ctxs, sd, p, 1)
    ms_s = timed(sequential)
    if g.genga_get_status(ctxs) != g.GENGA_OK:
        raise RuntimeError("device status after the sequential steps")
    ctxs.close()
    ms_b = max_over_ranks(ms_b, dist, dev)
    ms_bg = max_over_ranks(ms_bg, dist, dev)
    ms_s = max_over_ranks(ms_s, dist, dev)
    vb = weak_value(ws, pairs_step, K, ms_b)
    vs = weak_value(ws, pairs_step, K, ms_s)
    return {"workload": BATCH_WORKLOAD, "discs": len(ds), "bodies": int(sizes.sum()), "pairs_per_step": pairs_step,
            "steps": K, "value": vb, "unit": UNIT, "ms_per_step": ms_b / K, "sequential_value": vs,
            "sequential_ms_per_step": ms_s / K, "speedup_vs_sequential": vb / vs,
            "tuned_variant": bvar, "tuned_variant_shape": g.genga_kernel_variant_info(bvar) if bvar >= 0 else None,
            "variant_pass_ms": [round(v, 4) for v in bms],
            "graph_blocks": {"value": weak_value(ws, pairs_step, K, ms_bg), "ms_per_step": ms_bg / K,
                             "how": "genga_step_batched(.., 4): one captured CUDA graph per 4-step block"}}


# ----------------------------------------------------------------- TP2 ----
def run_tp2(g, torch, dev, stream, flush):
    """giants100k (4 giants + 100,000 planetesimals): the FP32 kick with every
    pair against test-particle mode 2 (planetesimals feel the giants only,
    the paper's setting for its giant-planet runs), and the FP64 mode-2 kick."""
    from paper_2309_08217_gb300 import discs
    d = discs.workload("giants100k")
    ctx = g.Context(d.N, dev.index)
    out = {"workload": "giants100k: 4 giants + 100,000 planetesimals (35 Earth masses) on 16-30 au, dt = 36.5 d",
           "n_big": 4}
    try:
        for label, nb, prec in (("fp32_all_pairs", -1, g.GENGA_FP32), ("fp32_tp2", 4, g.GENGA_FP32),
                                ("fp64_tp2", 4, g.GENGA_FP64)):
            p = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=prec, n_big=nb)
            s = g.DeviceSystem.from_disc(d, device=dev)
            for _ in range(3):
                g.genga_kick(ctx, s, p, 0.0, None)
            K = 5
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            torch.cuda.synchronize(dev)
            for k in range(K):
                flush.zero_()
                evs[k][0].record(stream)
                g.genga_kick(ctx, s, p, 0.0, None)
                evs[k][1].record(stream)
            torch.cuda.synchronize(dev)
            if g.genga_get_status(ctx) != g.GENGA_OK:
                raise RuntimeError("device status after the mode-2 kicks")
            out[label + "_kick_ms"] = sum(a.elapsed_time(b) for a, b in evs) / K
    finally:
        ctx.close()
    out["tp2_speedup_fp32"] = out["fp32_all_pairs_kick_ms"] / out["fp32_tp2_kick_ms"]
    return out


# --------------------------------------------------------------- genga ----
def run_genga(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2309_08217_gb300 as g
    from paper_2309_08217_gb300 import discs
    if rank == 0:
        g.build()
    if dist:
        dist.barrier()
    g.load()

    d = discs.disc_powerlaw(40_000, replica_seed(rank))  # rank 0: the disc40k workload itself
    N = d.N
    pairs_step = 2 * N * (N - 1)
    ctx = g.Context(N, local)
    p32 = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32)
    p64 = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP64)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    def timed_steps(params, K, W, clocks=False):
        s = g.DeviceSystem.from_disc(d, device=dev)
        for _ in range(W):
            g.genga_step(ctx, s, params, 1)
        if g.genga_get_status(ctx) != g.GENGA_OK:
            raise RuntimeError("device status after warm-up")
        g.genga_profile_enable(ctx, True)
        launches0 = g.genga_launch_count(ctx)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        sampler = ClockSampler(local) if clocks else None
        barrier()
        if sampler:
            sampler.start()
        for k in range(K):
            flush.zero_()                          # L2 flush between timed steps (not timed)
            evs[k][0].record(stream)
            g.genga_step(ctx, s, params, 1)
            evs[k][1].record(stream)
        barrier()
        clk = sampler.stop() if sampler else None
        st = g.genga_get_status(ctx)
        if st != g.GENGA_OK:
            raise RuntimeError(f"device status {st} after the timed steps")
        ms = sum(a.elapsed_time(b) for a, b in evs)
        pass_ms, launches = g.genga_profile_read(ctx)
        g.genga_profile_enable(ctx, False)
        timed_steps.kernels = g.genga_launch_count(ctx) - launches0
        return ms, pass_ms, launches, clk, s

    # ---- every FP32 pass variant on this workload (the autotuner keeps the fastest)
    variants = {}
    _, nvar = g.genga_get_kernel_variant(ctx, N)
    sv = g.DeviceSystem.from_disc(d, device=dev)
    for v in ([] if args.no_sweep else range(nvar)):
        g.genga_set_kernel_variant(ctx, v)
        for _ in range(2):
            g.genga_kick(ctx, sv, p32, 0.0, None)
        g.genga_profile_enable(ctx, True)
        for _ in range(5):
            g.genga_kick(ctx, sv, p32, 0.0, None)
        pms, pn = g.genga_profile_read(ctx)
        g.genga_profile_enable(ctx, False)
        variants[str(v)] = pms / max(1, pn)
    g.genga_set_kernel_variant(ctx, args.variant)
    g.genga_set_fp64_variant(ctx, args.fp64_variant)

    # ---- FP32 step (the headline) and FP64 step on the same GPU
    ms32, pass32, nl32, clk, s32 = timed_steps(p32, args.steps, args.warmup, clocks=True)
    kernels32 = timed_steps.kernels
    chosen, _ = g.genga_get_kernel_variant(ctx, N)
    tuner_ms = g.genga_tuning_times(ctx, N)
    ms64, pass64, nl64, _, _ = timed_steps(p64, max(1, args.fp64_steps), 3)
    chosen64, _ = g.genga_get_fp64_variant(ctx, N)
    tuner64_ms = g.genga_fp64_tuning_times(ctx, N)

    # ---- the 1,000-step run of the workload: mean step and pass times over the
    # whole run (the state evolves: the spatial order and the NEAR share drift)
    long_run = None
    if args.long_steps > 0:
        sl = g.DeviceSystem.from_disc(d, device=dev)
        g.genga_profile_enable(ctx, True)
        el0, el1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        el0.record(stream)
        g.genga_step(ctx, sl, p32, args.long_steps)
        el1.record(stream)
        barrier()
        lp_ms, lp_n = g.genga_profile_read(ctx)
        g.genga_profile_enable(ctx, False)
        if g.genga_get_status(ctx) != g.GENGA_OK:
            raise RuntimeError("device status after the long run")
        ms_long = max_over_ranks(el0.elapsed_time(el1), dist, dev)
        lp_avg = lp_ms / max(1, lp_n)
        long_run = {"steps": args.long_steps, "ms_per_step": ms_long / args.long_steps,
                    "value": weak_value(ws, pairs_step, args.long_steps, ms_long), "unit": UNIT,
                    "pass_ms_avg": lp_avg, "passes": lp_n,
                    "frac": FLOPS_PER_PAIR * N * (N - 1) / (lp_avg * 1e-3) / 1e12 / (
                        torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * 2070e6 / 1e12),
                    "how": "genga_step(ctx, sys, params, steps) from t = 0, one call, step by step (pass events on), "
                           "no L2 flush inside"}

    # ---- compaction of ghosts (mergers / removal): genga_compact on the
    # 40,000-body state with every 100th body a ghost (mass -0.0), with an id array
    compaction = None
    if args.bs_tol > 0:
        sc = g.DeviceSystem.from_disc(d, device=dev, radius=np.full(N, 1e-5))
        ids = torch.arange(N, dtype=torch.int32, device=dev)
        K = 10
        evc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        kept = 0
        for k in range(K + 2):
            for c in range(7):
                sc.tensors[c].copy_(torch.as_tensor(d.arrays()[c], device=dev))
            sc.radius.fill_(1e-5)
            sc.tensors[6][::100] = -0.0
            ids.copy_(torch.arange(N, dtype=torch.int32, device=dev))
            sc.c.N = N
            flush.zero_()
            if k >= 2:
                evc[k - 2][0].record(stream)
            kept = g.genga_compact(ctx, sc, ids)    # synchronises
            if k >= 2:
                evc[k - 2][1].record(stream)
        torch.cuda.synchronize(dev)
        ms_c = sorted(a.elapsed_time(b) for a, b in evc)[K // 2]
        moved = kept * (8 * 8 + 4) * 2 + N * 8      # read + write of the survivors (8 doubles, 1 int), masses scanned
        compaction = {"N": N, "ghosts": N - kept, "ms_median": ms_c, "moved_bytes": moved,
                      "GB_per_s": moved / (ms_c * 1e-3) / 1e9,
                      "how": "genga_compact (count, scan, scatter through a scratch, copy back), L2 flushed before "
                             "each call; the call synchronises, so the events also hold its host round trip"}

    # ---- the full hybrid step: the same FP32 steps with the close-encounter
    # (Bulirsch-Stoer) level on
    level1 = None
    if args.bs_tol > 0:
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        cap = 1 << 16
        pbuf = torch.zeros(2 * cap, dtype=torch.int32, device=dev)
        s1 = g.DeviceSystem.from_disc(d, device=dev)
        g.genga_kick(ctx, s1, p32, 0.0, None)
        g.genga_last_encounters(ctx, pbuf, cap, cnt)
        pairs0 = int(cnt.item())
        g.genga_get_status(ctx)          # (a list longer than cap only truncates this copy)
        p32_on = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32, bs_tol=args.bs_tol)
        ms_on, _, _, _, _ = timed_steps(p32_on, args.steps, args.warmup)
        ms_on = max_over_ranks(ms_on, dist, dev)
        level1 = {"bs_tol": args.bs_tol, "encounter_pairs_t0": pairs0,
                  "value_level_on": weak_value(ws, pairs_step, args.steps, ms_on), "unit": UNIT,
                  "ms_per_step_level_on": ms_on / args.steps,
                  "ms_per_step_level_off": max_over_ranks(ms32, dist, dev) / args.steps,
                  "how": "the headline FP32 steps again with the close-encounter level on: every group of "
                         "encounter pairs integrated by Bulirsch-Stoer over the drift"}

    def graph_blocks(params, blocks):
        """Steps as captured 4-step graphs (genga_step(.., 4)), L2 flushed between
        blocks; returns (max-over-ranks ms of all blocks, steps)."""
        sg = g.DeviceSystem.from_disc(d, device=dev)
        g.genga_step(ctx, sg, params, 8)          # aligns the order and captures the graph
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(blocks)]
        barrier()
        for k in range(blocks):
            flush.zero_()
            evb[k][0].record(stream)
            g.genga_step(ctx, sg, params, 4)
            evb[k][1].record(stream)
        barrier()
        if g.genga_get_status(ctx) != g.GENGA_OK:
            raise RuntimeError("device status after the graph blocks")
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evb), dist, dev), 4 * blocks

    # ---- intermediate levels of the changeover: the self-tuning call over a
    # few (levels, sub-steps), then the chosen setting timed like level1
    levels = None
    if args.bs_tol > 0 and not args.no_levels:
        cand = [(0, 2), (1, 2), (1, 4), (2, 2), (2, 3)]
        st = g.DeviceSystem.from_disc(d, device=dev)
        p32_on = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32, bs_tol=args.bs_tol)
        best, ms_c = g.genga_tune_levels(ctx, st, p32_on, cand, 8)
        if g.genga_get_status(ctx) != g.GENGA_OK:
            raise RuntimeError("device status after tuning the levels")
        chosen_lv = tuple(int(v) for v in args.levels.split(":")) if args.levels else best
        p32_lv = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32, bs_tol=args.bs_tol,
                               n_levels=chosen_lv[0], n_sub=chosen_lv[1])
        ms_lv, nsteps_lv = graph_blocks(p32_lv, max(1, args.steps // 4))
        p32_l0 = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32, bs_tol=args.bs_tol)
        ms_l0, _ = graph_blocks(p32_l0, max(1, args.steps // 4))
        levels = {"candidates": [list(c) for c in cand], "trial_ms_per_step": [round(v, 4) for v in ms_c],
                  "tuned": list(best), "timed": list(chosen_lv),
                  "value_timed": weak_value(ws, pairs_step, nsteps_lv, ms_lv), "unit": UNIT,
                  "ms_per_step_timed": ms_lv / nsteps_lv, "ms_per_step_no_levels": ms_l0 / nsteps_lv,
                  "how": "genga_tune_levels: 8 trial steps of each (n_levels, n_sub) from a copy of the state "
                         "(graph-launched, L2 not flushed); then the fastest (or --levels) and the level-1 step "
                         "without levels, both as captured 4-step graphs with L2 flushed between blocks"}
        # a dense group: a 10 Earth-mass planet with 80 planetesimals within 0.05 au, in a
        # 4,000-body disc (one 85-member close-encounter group), where Bulirsch-Stoer alone is slow
        dsw = discs.workload("swarm4k")
        csw = g.Context(dsw.N, local)
        ssw = g.DeviceSystem.from_disc(dsw, device=dev)
        psw = g.make_params(G=dsw.G, Mstar=dsw.Mstar, dt=dsw.dt, precision=g.GENGA_FP32, bs_tol=args.bs_tol)
        cand_sw = [(0, 2), (1, 4), (1, 8), (2, 3), (2, 4)]
        codes_sw = []
        best_sw, ms_sw = g.genga_tune_levels(csw, ssw, psw, cand_sw, 4, codes=codes_sw)
        if g.genga_get_status(csw) != g.GENGA_OK:
            raise RuntimeError("device status after tuning the levels on swarm4k")
        csw.close()
        pairs_sw = 2 * dsw.N * (dsw.N - 1)
        ms_best = ms_sw[cand_sw.index(best_sw)]
        levels["swarm4k"] = {
            "N": dsw.N, "candidates": [list(c) for c in cand_sw], "trial_ms_per_step": [round(v, 4) for v in ms_sw],
            "trial_status": codes_sw, "tuned": list(best_sw), "value_tuned": pairs_sw / (ms_best * 1e-3),
            "unit": UNIT, "speedup_over_no_levels": ms_sw[0] / ms_best,
            "how": "genga_tune_levels, 4 graph-launched trial steps per candidate from the same state; a "
                   "candidate whose trial raised a status (7: the Bulirsch-Stoer level hit its sub-step or "
                   "time limits and finished on Kepler orbits) is not chosen"}

    # ---- the same FP32 steps launched as captured 4-step graphs (genga_step(.., 4)),
    # L2 flushed between blocks
    blocks = max(1, args.steps // 4)
    sgr = g.DeviceSystem.from_disc(d, device=dev)
    g.genga_step(ctx, sgr, p32, 8)                # aligns the order and captures the graph
    evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(blocks)]
    barrier()
    for k in range(blocks):
        flush.zero_()
        evg[k][0].record(stream)
        g.genga_step(ctx, sgr, p32, 4)
        evg[k][1].record(stream)
    barrier()
    if g.genga_get_status(ctx) != g.GENGA_OK:
        raise RuntimeError("device status after the graph blocks")
    ms_graph = max_over_ranks(sum(a.elapsed_time(b) for a, b in evg), dist, dev)
    graph = {"value": weak_value(ws, pairs_step, 4 * blocks, ms_graph), "unit": UNIT,
             "ms_per_step": ms_graph / (4 * blocks), "steps": 4 * blocks,
             "how": "genga_step(ctx, sys, params, 4): one captured CUDA graph per 4-step block, "
                    "L2 flushed between blocks"}

    ms32_max = max_over_ranks(ms32, dist, dev)
    ms64_max = max_over_ranks(ms64, dist, dev)
    value = weak_value(ws, pairs_step, args.steps, ms32_max)
    value64 = weak_value(ws, pairs_step, max(1, args.fp64_steps), ms64_max)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in d.arrays()]
        outh = [torch.empty_like(host[c]).pin_memory() for c in range(6)]
        s = g.DeviceSystem.from_disc(d, device=dev)
        for _ in range(max(3, args.warmup)):
            g.genga_step(ctx, s, p32, 1)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            for c in range(7):
                s.tensors[c].copy_(host[c], non_blocking=True)
            g.genga_step(ctx, s, p32, 1)
            for c in range(6):
                outh[c].copy_(s.tensors[c], non_blocking=True)
        e1.record(stream)
        barrier()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": weak_value(ws, pairs_step, args.steps, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(h.numel() * 8 for h in host)),
               "d2h_bytes_per_step": int(sum(h.numel() * 8 for h in outh)),
               "ms_per_step": ms_e2e / args.steps}

    # ---- roofline of the dominant kernel (the FP32 long-range pass)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    peak32 = sms * 128 * 2 * max_mhz * 1e6 / 1e12            # FP32 CUDA-core FMA peak, TFLOP/s
    f32_meas, f64_meas = g.genga_measure_alu_peaks(local)
    f32x2_meas = g.genga_measure_fma2_peak(local)
    pass_avg = pass32 / max(1, nl32)
    pass64_avg = pass64 / max(1, nl64)
    achieved = FLOPS_PER_PAIR * N * (N - 1) / (pass_avg * 1e-3) / 1e12
    achieved64 = FLOPS_PER_PAIR * N * (N - 1) / (pass64_avg * 1e-3) / 1e12
    info = g.genga_kernel_variant_info(chosen) if chosen >= 0 else {"kind": 0}
    kname = "pass_mutual_kernel" if info["kind"] == 1 else "pass_fp32_kernel"
    traffic = kernel_traffic(kname)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32,
            "traffic": traffic, "kernel": kname, "variant_shape": info,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flops x {max_mhz:.0f} MHz",
            "flops_per_pair": FLOPS_PER_PAIR, "pass_ms_avg": pass_avg,
            "measured_ffma_tflops": f32_meas, "frac_of_measured_ffma": achieved / f32_meas,
            "measured_ffma2_tflops": f32x2_meas,
            "sm_mhz_median": (clk or {}).get("sm_mhz"), "fp32_variant": chosen,
            "fp32_variant_pass_ms": variants, "autotuner_pass_ms": tuner_ms}

    # ---- batched: 256 independent discs in one call vs one call per disc
    batched = None
    if not args.no_batched:
        batched = run_batched(g, torch, dev, stream, flush, args, rank, ws, dist)

    tp2 = None if args.no_tp2 else run_tp2(g, torch, dev, stream, flush)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # acc rows of the GPU FP32 kick for the sampled bodies (accuracy of this very run)
        sg = g.DeviceSystem.from_disc(d, device=dev)
        acc = torch.zeros(3 * N, dtype=torch.float64, device=dev)
        g.genga_kick(ctx, sg, p32, 0.0, acc)
        gacc = acc.view(3, N).cpu().numpy()
        rate, rows, thr, oacc, idx, el = oracle_sample_rate(d, args.cpu_seconds)
        err = np.sqrt(((gacc[:, idx] - oacc) ** 2).sum(0)) / np.sqrt((oacc ** 2).sum(0))
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"FP64 oracle pair sum over {rows} random body rows x {N - 1} partners ({el:.1f} s)",
               "fp32_rel_err_max_on_sample": float(err.max())}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "pairs_per_step": pairs_step,
                   "step": "kick(dt/2) drift(dt) kick(dt/2) via genga_step (the level-0 step); FP32 pair "
                           "terms, FP64 accumulation, FP64 drift and close-encounter pairs; the step with the "
                           "close-encounter level is in level1",
                   "l2": "flushed (512 MiB write) between timed steps, outside the step events",
                   "parallelism": f"{ws} independent replica disc(s), one per GPU"},
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64_max / max(1, args.fp64_steps),
                 "steps": max(1, args.fp64_steps), "pass_ms_avg": pass64_avg, "achieved_tflops": achieved64,
                 "measured_dfma_tflops": f64_meas, "frac_of_measured_dfma": achieved64 / f64_meas,
                 "fp32_over_fp64": value / value64, "fp64_variant": chosen64,
                 "kernel": "pass_mutual64_kernel" if chosen64 > 0 else "pass_fp64_kernel",
                 "variant_shape": g.genga_fp64_variant_info(chosen64) if chosen64 >= 0 else None,
                 "autotuner_pass_ms": tuner64_ms,
                 "traffic": kernel_traffic("pass_mutual64_kernel" if chosen64 > 0 else "pass_fp64_kernel")},
        "roofline": roof,
        "graph_blocks": graph,
        "long_run": long_run,
        "level1": level1,
        "levels": levels,
        "compaction": compaction,
        "batched": batched,
        "tp2": tp2,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": kernels32,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- conservation ----
def run_conservation(args):
    """Relative energy error and |dL/L| along FP32-kick and FP64-kick runs from
    the same seeded state (one JSON line per workload), both with the
    close-encounter level at --bs-tol (0: every body on its Kepler orbit, the
    (1 - K) part of encounter pairs then left out on both sides)."""
    import numpy as np
    import torch

    import paper_2309_08217_gb300 as g
    from paper_2309_08217_gb300 import discs
    g.build()
    g.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    for spec in args.conservation.split(","):
        fields = spec.split(":")
        name, steps, every = fields[0], int(fields[1]), int(fields[2])
        n_big = int(fields[3]) if len(fields) > 3 else -1   # test-particle mode 2 with n_big big bodies
        d = discs.workload(name)
        ctx = g.Context(d.N, 0)
        out = {"mode": "conservation", "workload": name, "N": d.N, "dt": d.dt, "steps": steps,
               "sample_every": every, "data": "synthetic", "bs_tol": args.bs_tol, "n_big": n_big}
        # per-body error of the FP32 kick against the FP64 kick at t = 0
        accs = []
        for prec in (g.GENGA_FP32, g.GENGA_FP64):
            p = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=prec, n_big=n_big)
            s = g.DeviceSystem.from_disc(d, device=dev)
            acc = torch.zeros(3 * d.N, dtype=torch.float64, device=dev)
            g.genga_kick(ctx, s, p, 0.0, acc)
            accs.append(acc.view(3, d.N).cpu().numpy())
        num = np.sqrt(((accs[0] - accs[1]) ** 2).sum(0))
        den = np.sqrt((accs[1] ** 2).sum(0))
        rel = num[den > 0] / den[den > 0]
        out["fp32_kick_rel_err_vs_fp64"] = {"max": float(rel.max()), "median": float(np.median(rel)),
                                             "p99": float(np.quantile(rel, 0.99))}
        for label, prec in (("fp32", g.GENGA_FP32), ("fp64", g.GENGA_FP64)):
            p = g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=prec, bs_tol=args.bs_tol, n_big=n_big)
            s = g.DeviceSystem.from_disc(d, device=dev)
            E0, *L0 = g.genga_energy(ctx, s, p)
            L0 = np.array(L0)
            dE, dLmag, dLvec = [], [], []
            t_ms = 0.0
            done = 0
            while done < steps:
                k = min(every, steps - done)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.genga_step(ctx, s, p, k)
                e1.record()
                torch.cuda.synchronize(dev)
                t_ms += e0.elapsed_time(e1)
                done += k
                E, *L = g.genga_energy(ctx, s, p)
                L = np.array(L)
                dE.append(E / E0 - 1.0)
                dLmag.append(np.linalg.norm(L) / np.linalg.norm(L0) - 1.0)
                dLvec.append(np.linalg.norm(L - L0) / np.linalg.norm(L0))
            st = g.genga_get_status(ctx)
            out[label] = {"dE_E_final": dE[-1], "dE_E_max_abs": float(np.max(np.abs(dE))),
                          "dL_L_final": dLmag[-1], "dL_L_max_abs": float(np.max(np.abs(dLmag))),
                          "dLvec_L_max": float(np.max(dLvec)), "ms_per_step": t_ms / steps, "status": st,
                          "dE_E_series": [float(v) for v in dE]}
        out["fp32_over_fp64_dL"] = out["fp32"]["dLvec_L_max"] / max(out["fp64"]["dLvec_L_max"], 1e-300)
        out["fp32_over_fp64_dE"] = out["fp32"]["dE_E_max_abs"] / max(out["fp64"]["dE_E_max_abs"], 1e-300)
        print(json.dumps(out), flush=True)
        ctx.close()
    return 0


def main():
    args = parse()
    if args.conservation:
        return run_conservation(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_genga(args)


if __name__ == "__main__":
    sys.exit(main())
