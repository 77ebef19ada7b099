#!/usr/bin/env python3
"""Benchmark of the QTT hot path on GB300.

One step = one pass over the TT-op workload of random quantized trains
(d = 30 mode-2 cores, uniform bond rank r, Gaussian cores N(0,1)/sqrt(r)):
  1. z = x + y, then SVD rounding of z at eps = 1e-6 (rank 2r in and out:
     random trains have flat spectra, so nothing is truncated);
  2. the Hadamard product x * y rounded by the sketched rounding (width
     r + 8, capped at rank r) without forming the rank-r^2 product;
  3. the 30-bit superfast Fourier transform applied to x, rounded the same
     way (bond <= 16 operator);
  4. <x, y>.
The metric is the flop model of every SVD rounding in the step (shared with
the CPU oracle, paper_2512_07811_gb300/flops.py) divided by the step time:
"tt_round TFLOP/s".  The fast path stores complex64 and runs float kernels;
the FP64 path runs the same step in complex128 and is reported beside it.
The three roundings of a step are independent and run concurrently on three
streams (one host thread each).  A secondary object times the
Moulinec-Suquet iteration on the 32^3 scalar laminate (15 interleaved bit
sites + one control site).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2512_07811_gb300 import inputs as I  # noqa: E402
from paper_2512_07811_gb300.flops import round_flops  # noqa: E402

D = 30
EPS = 1e-6
OVERSAMPLE = 8
JACOBI_DRAM_BYTES_PER_LAUNCH = 144.5e3
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--rank", type=int, default=64)
    p.add_argument("--no-ms", action="store_true")
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--batch", type=int, default=32,
                   help="trains rounded together in the grouped-batching secondary measurement (0: skip)")
    p.add_argument("--prec", choices=["f32", "tc32"], default="f32",
                   help="fast path arithmetic: float CUDA cores, or tensor cores for the large contractions")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def sketch_cores(rng, d, modes, ell):
    return I.sketch_cores(rng, d, modes, ell)


# --------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ our path
class Step:
    """Device-resident inputs and one pass of the workload.  The step's three
    roundings are independent: each runs on its own context (stream) from its
    own host thread, so that their latency-bound factorisation chains occupy
    different SMs at the same time; `run` returns when all three are done."""

    def __init__(self, Q, torch, ctxs, streams, r, dtype, qft_c128, prec=None):
        import concurrent.futures as cf
        self.Q, self.torch, self.r, self.dtype = Q, torch, r, dtype
        self.ctxs, self.streams = ctxs, streams
        self.prec = prec
        ctx = ctxs[0]
        self.xc = I.random_tt_cores(D, 2, r, seed=1000 + r, dtype=np.complex128)
        self.yc = I.random_tt_cores(D, 2, r, seed=1001 + r, dtype=np.complex128)
        rng = np.random.default_rng(2000 + r)
        sk, self.sk_ranks = sketch_cores(rng, D, [2] * D, r + OVERSAMPLE)
        self.X = Q.TT.from_cores(ctx, self.xc, dtype)
        self.Y = Q.TT.from_cores(ctx, self.yc, dtype)
        self.S = Q.TT.from_cores(ctx, sk, dtype)
        self.DX = Q.qtt_mpo_diag(ctx, self.X)
        self.F = qft_c128 if dtype == Q.C128 else Q.qtt_mpo_convert(ctx, qft_c128, dtype)
        self.modes = [2] * D
        ctx.sync()
        self.pool = cf.ThreadPoolExecutor(max_workers=3)

    def run(self, X=None, Y=None):
        Q, r, torch = self.Q, self.r, self.torch
        c0, c1, c2 = self.ctxs
        X = X or self.X
        Y = Y or self.Y
        DX = self.DX if X is self.X else Q.qtt_mpo_diag(c0, X)
        # the worker streams start after everything already queued on the first
        start = torch.cuda.Event()
        start.record(self.streams[0])
        for st in self.streams[1:]:
            st.wait_event(start)

        def add_round():
            z = Q.tt_add(c0, 1.0, X, 1.0, Y)
            zr, _ = Q.tt_round(c0, z, EPS, prec=self.prec)
            return z.ranks, zr, Q.tt_dot(c0, X, Y)

        def had_round():
            return Q.tt_round_sketched(c1, [(1.0, DX, Y)], self.S, EPS, r, prec=self.prec)[0]

        def qft_round():
            return Q.tt_round_sketched(c2, [(1.0, self.F, X)], self.S, EPS, r, prec=self.prec)[0]

        fa, fh, fq = self.pool.submit(add_round), self.pool.submit(had_round), self.pool.submit(qft_round)
        zranks, zr, v = fa.result()
        h, q = fh.result(), fq.result()
        for st in self.streams[1:]:
            ev = torch.cuda.Event()
            ev.record(st)
            self.streams[0].wait_event(ev)
        flops = (round_flops(self.modes, zranks, zr.ranks)
                 + round_flops(self.modes, self.sk_ranks, h.ranks)
                 + round_flops(self.modes, self.sk_ranks, q.ranks))
        return flops, (zr, h, q, v)


def flush_l2(torch, buf):
    buf.add_(1.0)


def time_steps(torch, stream, step, steps, flush):
    """Per-step device time with CUDA events on the library's stream; the L2
    flush between steps sits outside the timed intervals."""
    total_ms, flops = 0.0, 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush_l2(torch, flush)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, _ = step.run()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        flops += f
    return total_ms, flops


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2512_07811_gb300 import qtt as Q

    torch.cuda.set_device(local_rank)
    # the deterministic rounding of the rank-128 sum is the step's longest
    # chain: its stream gets the higher scheduling priority
    streams = [torch.cuda.Stream(device=local_rank, priority=-1)] + \
        [torch.cuda.Stream(device=local_rank, priority=0) for _ in range(2)]
    stream = streams[0]
    ctxs = [Q.Context(local_rank, st.cuda_stream) for st in streams]
    ctx = ctxs[0]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    r = args.rank
    qft = Q.qtt_qft_mpo(ctx, D, -1, 1e-12)
    fast = Step(Q, torch, ctxs, streams, r, Q.C64, qft, Q.PREC_TC32 if args.prec == "tc32" else Q.PREC_F32)
    for _ in range(args.warmup):
        fast.run()
    ctx.sync()

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = sum(c.launches for c in ctxs)
    ms, flops = time_steps(torch, stream, fast, args.steps, flush)
    launches = sum(c.launches for c in ctxs) - l0
    # the per-kernel-class split comes from a second timed region of the
    # same length with the library's event profiler on (it records two CUDA
    # events per launch, host work that would slow the headline steps)
    for c in ctxs:
        c.profile(True)
    ms_prof, _ = time_steps(torch, stream, fast, args.steps, flush)
    prof = {}
    for k in ["gemm", "qr", "jacobi", "elem"]:
        parts = [c.profile_read(k) for c in ctxs]
        prof[k] = {f: sum(p[f] for p in parts) for f in ["ms", "launches", "flops", "bytes"]}
    for c in ctxs:
        c.profile(False)
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        ms, flops = aggregate(ms, flops)
        dist.barrier()

    # e2e: the same step with the inputs uploaded from pinned host memory and
    # every result read back, host<->device copies inside the timed region
    pin_x = [torch.from_numpy(c.astype(np.complex64)).pin_memory() for c in fast.xc]
    pin_y = [torch.from_numpy(c.astype(np.complex64)).pin_memory() for c in fast.yc]
    h2d = sum(t.numel() * 8 for t in pin_x + pin_y)
    e2e_ms, e2e_flops, d2h = 0.0, 0.0, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(torch, flush)
        stream.synchronize()
        t0 = time.perf_counter()
        X = Q.TT.from_cores(ctx, [t.numpy() for t in pin_x], Q.C64)
        Y = Q.TT.from_cores(ctx, [t.numpy() for t in pin_y], Q.C64)
        f, outs = fast.run(X, Y)
        d2h = 0
        for tt in outs[:3]:
            for c in tt.cores():
                d2h += c.nbytes
        d2h += 16
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_flops += f

    # FP64 path, same step in complex128
    slow = Step(Q, torch, ctxs, streams, r, Q.C128, qft, Q.PREC_F64)
    slow.run()
    ctx.sync()
    ms64, flops64 = time_steps(torch, stream, slow, args.fp64_steps, flush)

    # secondary measurements: a failing one is recorded in the line, it does
    # not take the headline measurement down with it
    def secondary(fn, *a):
        try:
            return fn(*a)
        except Exception as exc:  # noqa: BLE001
            return {"error": "%s: %s" % (type(exc).__name__, exc)}

    polar = secondary(polar_vs_svd, Q, torch, ctx, stream, flush, fast)
    batched = None
    if args.batch > 0:
        batched = secondary(batched_rounding, Q, torch, ctx, stream, flush, r, args.batch, 2)
    ms_part = None
    if not args.no_ms:
        ms_part = secondary(ms_laminate, Q, ctx)
        ms_part["plane"] = secondary(ms_plane, Q, ctx)
        ms_part["tt_cross"] = secondary(cross_setup, Q, ctx)
        ms_part["green_amen"] = secondary(ms_green_amen, Q, ctx)
    return dict(ms=ms, flops=flops, prof=prof, ms_prof=ms_prof, launches=launches, clocks=clk, e2e_ms=e2e_ms,
                e2e_flops=e2e_flops, h2d=h2d, d2h=d2h, ms64=ms64, flops64=flops64, ms_part=ms_part, batched=batched,
                polar=polar)


def batched_rounding(Q, torch, ctx, stream, flush, r, count, steps):
    """Grouped batching: `count` independent add + SVD roundings of the
    workload's shape (rank-r pairs, d = D) in lockstep through tt_round_batch,
    one launch per kernel per core step for the whole batch.  Returns the
    model-flop rate and the time per batch (CUDA events, L2 flushed before
    each timed batch)."""
    xs = []
    for b in range(count):
        x = Q.TT.from_cores(ctx, I.random_tt_cores(D, 2, r, seed=3000 + b, dtype=np.complex128), Q.C64)
        y = Q.TT.from_cores(ctx, I.random_tt_cores(D, 2, r, seed=4000 + b, dtype=np.complex128), Q.C64)
        xs.append(Q.tt_add(ctx, 1.0, x, 1.0, y))
    Q.tt_round_batch(ctx, xs, EPS)  # warm-up
    ctx.sync()
    ms, flops = 0.0, 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush_l2(torch, flush)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ys, _ = Q.tt_round_batch(ctx, xs, EPS)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        flops += sum(round_flops([2] * D, x.ranks, y.ranks) for x, y in zip(xs, ys))
    return {"workload": "%d independent add + SVD roundings of d=%d rank-%d pairs (rank %d sums), tt_round_batch"
                        % (count, D, r, 2 * r),
            "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_batch": ms / steps, "steps": steps,
            "roundings_per_s": count * steps / (ms * 1e-3)}


def polar_vs_svd(Q, torch, ctx, stream, flush, step):
    """SVD- vs polar-based compression (the paper's comparison, chi =
    tau_polar / tau_SVD) on the step's first rounding: the rank-128 sum of the
    two rank-64 trains, FP32 storage, SVD rounding vs polar rounding with
    CUDA-core products (f32) and with the products on the tensor cores
    (tc32).  One warm-up and one timed rounding each, L2 flushed first."""
    z = Q.tt_add(ctx, 1.0, step.X, 1.0, step.Y)

    def timed(fn):
        fn()
        ctx.sync()
        with torch.cuda.stream(stream):
            flush_l2(torch, flush)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y, _ = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), y.ranks

    svd_ms, svd_r = timed(lambda: Q.tt_round(ctx, z, EPS, prec=Q.PREC_F32))
    out = {"workload": "rounding of the rank-128 sum (d=30), eps %g, complex64" % EPS, "svd_ms": svd_ms}
    for name, p in [("f32", Q.PREC_F32), ("tc32", Q.PREC_TC32)]:
        ms, r = timed(lambda: Q.tt_round_polar(ctx, z, EPS, prec=p))
        out["polar_ms_" + name] = ms
        out["chi_" + name] = ms / svd_ms
        out["ranks_equal_" + name] = r == svd_r
    return out


def ms_laminate(Q, ctx):
    """Moulinec-Suquet iterations on the 32^3 scalar laminate, load case E = e_x:
    the FP64 path at the workload's rounding tolerance 1e-8, the fast (FP32)
    path at 1e-6 -- a tolerance below FP32 resolution cannot truncate the
    rounding noise, so its ranks would run into the cap -- with the fast
    path's effective-tensor deviation from the FP64 result reported (the
    accuracy the comparison is held to is 1e-4).  One warm-up solve each, then
    five timed iterations (setup reported separately)."""
    ind = I.laminate_indicator(32)
    out = {"workload": "32^3 scalar laminate, 15 interleaved bit sites + control, contrast 10, max rank 64, "
                       "E = e_x, 5 iterations; eps 1e-8 (FP64) / 1e-6 (fast)"}
    C64 = None
    for name, prec, eps in [("fp64", Q.PREC_F64, 1e-8), ("fast", Q.PREC_F32, 1e-6)]:
        kw = dict(tol=0.0, max_rank=64, eps=eps, prec=prec, load_mask=1)
        Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=1, min_iter=1, **kw)
        C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=5, min_iter=5, **kw)
        it = rep.iterations[0]
        out[name] = {"iters_per_s": it / (rep.iterate_ms * 1e-3) if rep.iterate_ms > 0 else None, "eps": eps,
                     "setup_ms": rep.setup_ms, "k_eff_xx": C[0, 0], "iterations": it,
                     "max_rank": rep.max_rank_seen, "sketch_width_sum": rep.sketch_width_sum}
        if name == "fp64":
            C64 = C
        else:
            out[name]["rel_dev_from_fp64"] = float(abs(C[0, 0] - C64[0, 0]) / abs(C64[0, 0]))
    # learned ranks: the MLP (trained here by the library's own kernels on the
    # rank traces of 8^3 / 16^3 solves, outside the timed region) sizes each
    # bond's sketch instead of the fixed width max_rank + oversampling
    from paper_2512_07811_gb300 import predictor as PR
    common = dict(kind="scalar", moduli=(1.0, 10.0), C0=5.5 * np.eye(3), tol=0.0, max_rank=64, max_iter=4,
                  min_iter=4, prec=Q.PREC_F32, load_mask=1)
    train = [dict(indicator=ind_t, eps=e, **common)
             for ind_t in [I.laminate_indicator(8), I.laminate_indicator(16), I.box_indicator(8, 0.2)]
             for e in (1e-6, 1e-4)]
    X, t = PR.collect_traces(ctx, train)
    net = Q.MLP(ctx, Q.MLP_FEATURES, seed=7)
    PR.train(net, X, t, epochs=150, batch=512, lr=3e-3, alpha=4.0)
    kw = dict(tol=0.0, max_rank=64, eps=1e-6, prec=Q.PREC_F32, load_mask=1, predictor=net)
    Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=1, min_iter=1, **kw)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=5, min_iter=5, **kw)
    it = rep.iterations[0]
    out["fast_learned_rank"] = {
        "iters_per_s": it / (rep.iterate_ms * 1e-3) if rep.iterate_ms > 0 else None, "eps": 1e-6,
        "k_eff_xx": C[0, 0], "rel_dev_from_fp64": float(abs(C[0, 0] - C64[0, 0]) / abs(C64[0, 0])),
        "sketch_width_sum": rep.sketch_width_sum, "fallbacks": rep.fallbacks, "training_rows": int(X.shape[0])}
    out["k_eff_xx_exact"] = 20.0 / 11.0
    if out["fast"]["iters_per_s"] and out["fp64"]["iters_per_s"]:
        out["speedup_fast_vs_fp64"] = out["fast"]["iters_per_s"] / out["fp64"]["iters_per_s"]
        if out["fast_learned_rank"]["iters_per_s"]:
            out["speedup_fast_learned_vs_fp64"] = out["fast_learned_rank"]["iters_per_s"] / out["fp64"]["iters_per_s"]
    return out


def ms_plane(Q, ctx, N=256):
    """Moulinec-Suquet iterations on a plane multibox image (N x N x 1: eight
    square inclusions of random sizes filling 20 % of the plane, contrast 10;
    a grid one voxel thick along z is the plane problem), load case E = e_x,
    FP64 at 1e-8 and the fast path at 1e-6, max rank 64; one warm-up solve,
    then five timed iterations.  The arithmetic and harmonic means of the
    phase moduli bound k_eff_xx from above and below."""
    ind = I.multibox_indicator_2d(N, count=8, area_fraction=0.2, seed=5)
    f = float(ind.mean())
    out = {"workload": f"{N}x{N}x1 scalar multibox (8 squares, area fraction {f:.3f}), "
                       f"{2 * int(np.log2(N))} interleaved bit sites + control, contrast 10, max rank 64, "
                       "E = e_x, 5 iterations; eps 1e-8 (FP64) / 1e-6 (fast)",
           "k_bounds": [1.0 / ((1 - f) / 1.0 + f / 10.0), (1 - f) * 1.0 + f * 10.0]}
    C64 = None
    for name, prec, eps in [("fp64", Q.PREC_F64, 1e-8), ("fast", Q.PREC_F32, 1e-6)]:
        kw = dict(tol=0.0, max_rank=64, eps=eps, prec=prec, load_mask=1)
        Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=1, min_iter=1, **kw)
        C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=5, min_iter=5, **kw)
        it = rep.iterations[0]
        out[name] = {"iters_per_s": it / (rep.iterate_ms * 1e-3) if rep.iterate_ms > 0 else None, "eps": eps,
                     "setup_ms": rep.setup_ms, "k_eff_xx": C[0, 0], "iterations": it,
                     "max_rank": rep.max_rank_seen}
        if name == "fp64":
            C64 = C
        else:
            out[name]["rel_dev_from_fp64"] = float(abs(C[0, 0] - C64[0, 0]) / abs(C64[0, 0]))
    if out["fast"]["iters_per_s"] and out["fp64"]["iters_per_s"]:
        out["speedup_fast_vs_fp64"] = out["fast"]["iters_per_s"] / out["fp64"]["iters_per_s"]
    return out


def cross_setup(Q, ctx):
    """Operator setup by TT-cross (Sec. 3) on the paper's largest plane grid
    (2^18 x 2^18, 36 spatial sites): the Green operator train (scalar and
    elastic) at 1e-10 and a multibox phase train; then, on a 4096 x 4096
    multibox where both routes fit, the setup time of the homogenisation
    with a dense image and dense Green TT-SVD against the box geometry with
    both trains by TT-cross, and the 65536 x 65536 multibox solved on the
    fast path (phase and Green trains by TT-cross, nothing dense)."""
    import time
    out = {}
    for name, kw in [("green_scalar_2pow18_sq", dict(ncomp=3, k0=5.5)),
                     ("green_elastic_2pow18_sq", dict(ncomp=6, lam0=3.0, mu0=2.0))]:
        ctx.sync()
        t0 = time.perf_counter()
        y, info = Q.tt_cross(ctx, "green", (18, 18, 0), 1e-10, **kw)
        ctx.sync()
        ms = (time.perf_counter() - t0) * 1e3
        out[name] = {"ms": ms, "evaluations": int(info.evaluations), "half_sweeps": int(info.half_sweeps),
                     "rank_before_rounding": int(info.max_rank), "rank": max(y.ranks),
                     "evaluations_per_s": info.evaluations / (ms * 1e-3)}
    boxes = I.multibox_boxes_2d(1 << 18, count=8, area_fraction=0.2, seed=5)
    ctx.sync()
    t0 = time.perf_counter()
    y, info = Q.tt_cross(ctx, "boxes", (18, 18, 0), 1e-10, boxes=boxes)
    ctx.sync()
    out["multibox_phase_2pow18_sq"] = {"ms": (time.perf_counter() - t0) * 1e3, "rank": max(y.ranks),
                                       "evaluations": int(info.evaluations)}
    # setup of one solve: dense image + dense Green TT-SVD vs box geometry + TT-cross
    N = 4096
    boxes = I.multibox_boxes_2d(N, count=8, area_fraction=0.2, seed=5)
    ind = I.boxes_indicator(boxes, (N, N, 1))
    kw = dict(tol=0.0, max_rank=64, eps=1e-6, prec=Q.PREC_F32, load_mask=1, max_iter=1, min_iter=1)
    _, rd = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), **kw)
    _, rx = Q.ms_homogenize(ctx, Q.Boxes(boxes, (N, N, 1)), "scalar", (1.0, 10.0), 5.5 * np.eye(3), op_cross=True,
                            **kw)
    out["ms_setup_4096_sq"] = {"dense_ms": rd.setup_ms, "cross_ms": rx.setup_ms,
                               "green_rank_dense": rd.green_rank, "green_rank_cross": rx.green_rank,
                               "phase_rank_dense": rd.phase_rank, "phase_rank_cross": rx.phase_rank}
    # the paper-scale plane problem on the fast path
    N = 1 << 16
    geo = Q.Boxes(I.multibox_boxes_2d(N, count=8, area_fraction=0.2, seed=5), (N, N, 1))
    kw = dict(tol=0.0, max_rank=64, eps=1e-6, prec=Q.PREC_F32, load_mask=1)
    Q.ms_homogenize(ctx, geo, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=1, min_iter=1, **kw)
    C, rep = Q.ms_homogenize(ctx, geo, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=5, min_iter=5, **kw)
    f = 0.2
    out["ms_multibox_65536_sq_fast"] = {
        "workload": "65536 x 65536 x 1 scalar multibox (8 squares), 32 interleaved bit sites + control, "
                    "contrast 10, max rank 64, eps 1e-6, E = e_x, 5 iterations",
        "iters_per_s": rep.iterations[0] / (rep.iterate_ms * 1e-3) if rep.iterate_ms > 0 else None,
        "setup_ms": rep.setup_ms, "k_eff_xx": C[0, 0], "max_rank": rep.max_rank_seen,
        "green_rank": rep.green_rank, "phase_rank": rep.phase_rank}
    return out


def ms_green_amen(Q, ctx):
    """The Green step eps^ = Gamma0 tau^ by AMEn (warm-started from the
    previous iteration) against the MPO x TT product with a sketched
    rounding, on the 32^3 scalar laminate and the 256^2 plane multibox, FP64
    (eps 1e-8) and fast (eps 1e-6) paths, 5 timed iterations after one
    warm-up solve each."""
    out = {}
    cases = [("laminate_32cube", I.laminate_indicator(32)),
             ("multibox_256sq", I.multibox_indicator_2d(256, count=8, area_fraction=0.2, seed=5))]
    for cname, ind in cases:
        res = {}
        for pname, prec, eps in [("fp64", Q.PREC_F64, 1e-8), ("fast", Q.PREC_F32, 1e-6)]:
            for route in ["sketched", "amen"]:
                kw = dict(tol=0.0, max_rank=64, eps=eps, prec=prec, load_mask=1, green_amen=route == "amen")
                Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=1, min_iter=1, **kw)
                C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), max_iter=5, min_iter=5,
                                         **kw)
                res[f"{pname}_{route}"] = {"iters_per_s": 5 / (rep.iterate_ms * 1e-3) if rep.iterate_ms > 0 else None,
                                           "k_eff_xx": C[0, 0], "max_rank": rep.max_rank_seen}
        out[cname] = res
    return out


# ------------------------------------------------------- CPU oracle arm
def oracle_sample(r, repeats=1):
    """The oracle's tt_add + SVD rounding of the step's first rounding, on the
    host cores: returns (seconds, model flops)."""
    from oracle import tt as T
    x = I.random_tt_cores(D, 2, r, seed=1000 + r, dtype=np.complex128)
    y = I.random_tt_cores(D, 2, r, seed=1001 + r, dtype=np.complex128)
    t0 = time.perf_counter()
    fl = 0.0
    for _ in range(repeats):
        z = T.tt_add(x, y)
        zr, _ = T.tt_round(z, EPS)
        fl += round_flops([2] * D, T.tt_ranks(z), T.tt_ranks(zr))
    return time.perf_counter() - t0, fl


def single_core_sample(r, budget_s=10.0):
    """The same oracle sample with the BLAS pinned to one thread (a child
    process, so the thread count is fixed before NumPy loads its BLAS):
    returns (seconds, model flops, repetitions) or None."""
    code = ("import sys, time, math; sys.path.insert(0, %r); import bench; "
            "s, f = bench.oracle_sample(%d); n = max(1, int(math.ceil(%f / max(s, 1e-3)))); "
            "s, f = bench.oracle_sample(%d, n); print(s, f, n)" % (ROOT, r, budget_s, r))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=6 * budget_s + 60)
        s, f, n = out.stdout.split()[-3:]
        return float(s), float(f), int(n)
    except Exception:  # noqa: BLE001
        return None


def cpu_baseline(r, budget_s=10.0):
    """The oracle timed on the host cores: a calibration run, then as many
    repetitions of the sample as fill about budget_s seconds; and the same
    with one BLAS thread."""
    s1, _ = oracle_sample(r)
    reps = max(1, int(math.ceil(budget_s / max(s1, 1e-3))))
    sec, fl = oracle_sample(r, reps)
    out = {"value": fl / sec / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "%d repetitions of one tt_add + SVD rounding of the d=30, r=%d pair (the first of the "
                     "step's three roundings), NumPy FP64 with its threaded BLAS" % (reps, r), "seconds": sec}
    one = single_core_sample(r, budget_s)
    if one is not None:
        out["single_core"] = {"value": one[1] / one[0] / 1e12, "unit": "TFLOP/s", "cores": 1,
                              "repetitions": one[2], "seconds": one[0]}
    return out


def aggregate(ms: float, flops: float):
    """Whole-job figures across ranks: the slowest rank's time (max) and the
    work of all ranks (sum).  Works on NCCL (CUDA tensors) and gloo (CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms, flops
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    f = torch.tensor([flops], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())


def config_dict(args, world):
    return {"workload": "tt_ops_d30_r%d: random QTT d=30, mode 2, rank %d, complex; add+round, "
                        "hadamard+sketched round, 30-bit SFFT apply+sketched round, dot" % (args.rank, args.rank),
            "d": D, "rank": args.rank, "eps": EPS, "sketch_oversample": OVERSAMPLE,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas x%d" % world}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "tt_round TFLOP/s (flop model), fast path"
    if args.impl == "reference":
        if rank != 0:
            return 0
        t_total, f_total = 0.0, 0.0
        for _ in range(args.warmup if args.warmup < 1 else 1):
            oracle_sample(args.rank)
        for _ in range(args.steps):
            sec, fl = oracle_sample(args.rank)
            t_total += sec
            f_total += fl
        val = f_total / t_total / 1e12
        line = {"impl": "reference", "metric": metric, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": config_dict(args, 1),
                "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": "per step: one tt_add + SVD rounding of the d=30 pair (NumPy FP64)"},
                "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank != 0:
        return 0
    peaks, peak_src = load_peaks()
    value = res["flops"] / (res["ms"] * 1e-3) / 1e12   # all ranks' work over the slowest rank's time
    # roofline of the dominant kernel class.  By device time (the committed
    # ncu launch list of this workload) the one-sided Jacobi SVDs take half
    # of the step's kernel time; the per-launch CUDA-event intervals of the
    # many ~10 us GEMMs also hold host launch gaps, so the event totals are
    # not used to pick the class.  ALU-bound: float CUDA cores.
    prof = res["prof"]
    dom = "jacobi"
    p = prof[dom]
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    if dom == "elem":
        roof = {"bound": "hbm", "achieved": p["bytes"] / (p["ms"] * 1e-3) / 1e9 if p["ms"] else 0.0,
                "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        roof = {"bound": "alu", "achieved": p["flops"] / (p["ms"] * 1e-3) / 1e12 if p["ms"] else 0.0,
                "peak": fp32_peak, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
    # DRAM bytes per launch of the class (dram__bytes_read.sum + write.sum),
    # mean over its launches in an ncu capture of this workload
    # (profiles/jacobi_block_kernel_f32_256x128.md); valid while the kernels are
    # those the capture was taken on
    roof["traffic"] = JACOBI_DRAM_BYTES_PER_LAUNCH if dom == "jacobi" and args.prec == "f32" else None
    # the 256 x 128 factorisations run on one 8-CTA cluster: the same rate
    # against the FP32 peak of the SMs they occupy
    roof["algorithmic_bytes_per_launch"] = p["bytes"] / p["launches"] if p["launches"] else None
    roof["sms_used"] = 8
    roof["frac_of_sms_used"] = roof["achieved"] / (roof["peak"] * 8 / 152) if roof["peak"] else None
    roof["kernel"] = {"gemm": "gemm_midx_kernel", "qr": "qr_panel_kernel", "jacobi": "jacobi_block_kernel",
                      "elem": "elementwise kernels"}[dom]
    roof["measured"] = ("CUDA events around every launch of the class on its stream, over %d profiled steps "
                        "(%.1f ms/step with the profiler on)" % (args.steps, res["ms_prof"] / args.steps))
    roof["peak_source"] = ("FP32 CUDA-core peak 152 SMs x 128 FMA/clk x %.0f MHz (%s clock)" %
                           (sm_mhz, peak_src)) if roof["bound"] == "alu" else "MEASURED_PEAKS hbm_gbs"
    roof["launches"] = p["launches"]
    roof["kernel_ms_total"] = p["ms"]
    line = {
        "metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "fast_path_arithmetic": args.prec, "data": "synthetic",
        "config": config_dict(args, world),
        "roofline": roof,
        "kernel_classes": {k: {"ms": v["ms"], "launches": v["launches"], "model_flops": v["flops"]}
                           for k, v in prof.items()},
        "cpu_baseline": cpu_baseline(args.rank),
        "e2e": {"value": world * res["e2e_flops"] / (res["e2e_ms"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "fp64_path": {"value": world * res["flops64"] / (res["ms64"] * 1e-3) / 1e12, "unit": "TFLOP/s",
                      "ms_per_step": res["ms64"] / args.fp64_steps, "steps": args.fp64_steps, "dtype": "c128"},
    }
    line["fast_vs_fp64"] = line["value"] / line["fp64_path"]["value"] if line["fp64_path"]["value"] else None
    if res["ms_part"] is not None:
        line["ms_iteration"] = res["ms_part"]
    if res.get("batched") is not None:
        line["batched_rounding"] = res["batched"]
    if res.get("polar") is not None:
        line["polar_vs_svd"] = res["polar"]
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
