#!/usr/bin/env python3
"""Throughput of the global registration hot path (Sec. IV, Algorithm 1, plus
the robust refinement) on GB300.

One step registers one fragment pair per GPU (pairs are independent, so N GPUs
run N replicas on N different pairs: weak scaling, no collective). The default
workload is the 150,000-point room pair on a 1 cm grid, FP32 end to end.
Inputs are resident in HBM when the timed region starts and L2 is flushed
(a 256 MB write) between steps, outside the timed events. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 0|1|2|3|4] [--match fp32|bf16|bf16_plain]
                  [--impl ours|reference]

--config 2 times the batched workload instead: 256 room pairs of 10k-120k
points per cloud registered by one lsr_register_batch call per step (BF16
tensor-core matching, concurrent streams, one CUDA graph), beside the plain
FP32 single-pair path on the same pairs. --config 3 does the same for 64
pairs of 200k points; --config 4 times the batched robust objective forward
and backward of 32 pairs of 50k points.

Under torchrun every rank runs its own pairs; the only collective is the
max over ranks of the timed region.

--match selects the descriptor matcher (FP32 SIMT, or the tensor-core matcher
with hi/lo or plain BF16 operands); every choice gives the same correspondences.

--impl reference times the FP64 CPU oracle (the only reference for this path)
on a bounded sample of the same workload, scaled to one pair.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fragment pairs/sec at ≤0.05°/≤0.5 mm vs plain FP32 path; HBM GB/s, TC util"
WORKLOADS = {
    0: "objects scene pair, 5,000 points per cloud, 70% overlap, 10% outliers, 4M hypotheses, FP32",
    1: "indoor room pair on a 1 cm voxel grid, 150,000 points per cloud, 50% overlap, 4M hypotheses, FP32",
    2: "256 indoor room pairs on a 1 cm voxel grid, 10k-120k points per cloud, 30-80% overlap, 4M hypotheses "
       "each, one batch per step (BF16 tensor-core matching, concurrent streams, one CUDA graph)",
    3: "64 indoor room pairs on a 1 cm voxel grid, 200,000 points per cloud, 50% overlap, 4M hypotheses each, "
       "one batch per step (BF16 tensor-core matching, FP32 re-rank of the 8 best 16-row candidate chunks, a superset "
       "of the top 8; concurrent streams, one CUDA graph)",
    4: "32 indoor room pairs of 50,000 points per cloud: robust alignment objective forward + backward (points and "
       "se(3) pose) for all pairs per step through RobustAlignBatch",
}
BATCH_PAIRS = {2: 256, 3: 64, 4: 32}
MATCH_MODES = {"fp32": 0, "bf16": 1, "bf16_plain": 2}
FP32_LANES_PER_SM = 128
N_SM = 152


# ---------------------------------------------------------------- ranks
def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: the job ends when its last rank does."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, total_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (every rank does the same amount of work: weak scaling)."""
    return world * units_per_rank / (total_ms * 1e-3)


def rank_pair_ids(config: int, rank: int) -> list:
    """The generator pair ids a rank registers in the batched configurations:
    disjoint blocks, so N ranks run N different batches."""
    n = BATCH_PAIRS[config]
    return list(range(rank * n, (rank + 1) * n))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device, self.proc, self.lines = device, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, sm_max_nominal):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": sm_max_nominal, "reasons": ["not sampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch

    import paper_1801_01572_gb300 as lsr
    from synth import make_pair

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    fp = make_pair(args.config, pair=rank, n_p=args.points, n_q=args.points)
    nP, nQ = len(fp.P), len(fp.Q)
    P = torch.from_numpy(fp.P).cuda()
    Q = torch.from_numpy(fp.Q).cuda()
    stream = torch.cuda.Stream()
    ctx = lsr.Context(dev, stream=stream.cuda_stream, match_precision=MATCH_MODES[args.match])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.register_pair(P, Q, fp.vpP, fp.vpQ)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    pk, _ = peaks()
    times, stages, last = [], np.zeros(8), None
    with ClockSampler(dev) as clk:
        l0 = lsr.launch_count()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = ctx.register_pair(P, Q, fp.vpP, fp.vpQ)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = lsr.launch_count() - l0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = float(sum(times))
    total_ms = max_over_ranks(total_ms, world)
    # per-stage device times (and the FP32 matcher's term count) from profiled
    # runs after the timed region: stage events and the counting matcher
    ctx.set_profiling(True)
    n_prof = min(args.steps, 3)
    for _ in range(n_prof):
        with torch.cuda.stream(stream):
            flush.zero_()
        prof = ctx.register_pair(P, Q, fp.vpP, fp.vpQ)
        stages += np.array(prof.stage_ms)
    ctx.set_profiling(False)
    stage_ms = stages / n_prof

    # end to end through the public API from pinned host memory
    Ph = torch.from_numpy(fp.P).pin_memory()
    Qh = torch.from_numpy(fp.Q).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        ctx.register_pair(Ph, Qh, fp.vpP, fp.vpQ)
    e2e_times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.register_pair(Ph, Qh, fp.vpP, fp.vpQ)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = float(sum(e2e_times))
    e2e_ms = max_over_ranks(e2e_ms, world)
    # the information matrix of eq. (5)-(6) of the registered pair (loop
    # verification; eps = 0.05 m as the paper), clouds resident, Q's grid built per call
    info_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, n_corr = ctx.information_matrix(P, Q, last.T, 0.05)
        e1.record(stream)
        e1.synchronize()
        info_ms.append(e0.elapsed_time(e1))
    # dense model correction of eq. (7) on a 2M-surfel room map and a 300-keyframe loop, resident
    # inputs; algorithmic bytes 32 in + 25 out per surfel
    from synth.surfels import make_surfels
    smap = make_surfels(2_000_000, 300, seed=3)
    sd = [torch.from_numpy(x).cuda() for x in (smap.pos, smap.nrm, smap.t0, smap.tu)]
    ctx.surfel_correct(*sd, smap.T_old, smap.T_new, smap.t_kf, smap.cam)
    surf_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, _, n_kept = ctx.surfel_correct(*sd, smap.T_old, smap.T_new, smap.t_kf, smap.cam)
        e1.record(stream)
        e1.synchronize()
        surf_ms.append(e0.elapsed_time(e1))
    # voxel downsampling of Algorithm 1 (5 cm leaf) of the resident P cloud; the means come back to the host
    vox_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        vox = ctx.voxel_downsample(P, 0.05)
        vox_ms.append((time.perf_counter() - t0) * 1e3)
    h2d, d2h = lsr.transfer_bytes(nP, nQ)
    info = dict(fp=fp, nP=nP, nQ=nQ, last=last, prof=prof, stage_ms=stage_ms, total_ms=total_ms, e2e_ms=e2e_ms, h2d=h2d,
                d2h=d2h, launches=launches, clocks=clk.summary(pk.get("sm_max_mhz")), peaks=pk,
                information={"ms": float(np.median(info_ms)), "correspondences": int(n_corr), "eps": 0.05},
                voxel={"ms": float(np.median(vox_ms)), "points": nP, "voxels": len(vox), "leaf": 0.05,
                       "note": "wall time of the call: key bounds, a host read of them, the cell pass, the copy back"},
                surfels={"ms": float(np.median(surf_ms)), "surfels": len(smap.pos), "keyframes": len(smap.t_kf),
                         "kept": int(n_kept),
                         "GB/s": 57.0 * len(smap.pos) / (float(np.median(surf_ms)) * 1e-3) / 1e9,
                         "note": "call time incl. the keyframe transforms' upload; 57 B per surfel"},
                params=ctx.params, match=args.match)
    ctx.close()

    # the other descriptor matchers on the same resident inputs (same result required)
    info["variants"] = {}
    if world == 1 and args.variants:
        for name in sorted(MATCH_MODES):
            if name == args.match:
                continue
            vctx = lsr.Context(dev, stream=stream.cuda_stream, match_precision=MATCH_MODES[name])
            vctx.set_profiling(True)
            for _ in range(args.warmup):
                vctx.register_pair(P, Q, fp.vpP, fp.vpQ)
            vt, vst, vl = [], np.zeros(8), None
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vl = vctx.register_pair(P, Q, fp.vpP, fp.vpQ)
                e1.record(stream)
                e1.synchronize()
                vt.append(e0.elapsed_time(e1))
                vst += np.array(vl.stage_ms)
            vctx.close()
            info["variants"][name] = {
                "value": args.steps / (sum(vt) * 1e-3), "unit": "pairs/s", "ms_per_step": sum(vt) / args.steps,
                "match_ms": float(vst[3] / args.steps), "match_fallbacks": vl.match_fallbacks,
                "identical_pose": bool(np.array_equal(vl.T, last.T)) and vl.inliers == last.inliers}
    return info


# ---------------------------------------------------------------- configs 2-4
def _gen_pair(ci):
    from synth import make_pair
    p = make_pair(*ci)
    return p.P, p.Q, p.vpP, p.vpQ, p.T


def batch_pairs(config, rank):
    """The pairs of this rank, generated in parallel host processes before any
    GPU work."""
    import multiprocessing as mp
    ids = [(config, i) for i in rank_pair_ids(config, rank)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_pair, ids, chunksize=2)


def _timed(stream, flush, fn):
    import torch
    with torch.cuda.stream(stream):
        flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_batch(args, rank, world, pairs):
    import torch

    import paper_1801_01572_gb300 as lsr

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    P = [torch.from_numpy(p[0]).cuda() for p in pairs]
    Q = [torch.from_numpy(p[1]).cuda() for p in pairs]
    vp = np.concatenate([np.concatenate([p[2], p[3]]) for p in pairs]).astype(np.float32)
    npts = sum(len(p[0]) + len(p[1]) for p in pairs)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ctx = lsr.Context(dev, stream=stream.cuda_stream, match_precision=MATCH_MODES["bf16"], batch_graph=1)
    for _ in range(args.warmup):  # the first call tunes tiles and streams, the next captures the graph
        res = ctx.register_batch(P, Q, vp)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    pk, _ = peaks()
    times = []
    with ClockSampler(dev) as clk:
        l0 = lsr.launch_count()
        for _ in range(args.steps):
            ms, res = _timed(stream, flush, lambda: ctx.register_batch(P, Q, vp))
            times.append(ms)
        launches = lsr.launch_count() - l0
    total_ms = float(sum(times))
    total_ms = max_over_ranks(total_ms, world)
    # end to end from pinned host memory (host-to-device copies inside the call)
    Ph = [torch.from_numpy(p[0]).pin_memory() for p in pairs]
    Qh = [torch.from_numpy(p[1]).pin_memory() for p in pairs]
    ctx.register_batch(Ph, Qh, vp)
    e2e = [_timed(stream, flush, lambda: ctx.register_batch(Ph, Qh, vp))[0] for _ in range(max(1, args.steps // 2))]
    e2e_ms = float(sum(e2e)) / len(e2e)
    ctx.close()
    # the plain FP32 single-pair path on the first pairs of the same batch
    m = min(32, len(pairs))
    sctx = lsr.Context(dev, stream=stream.cuda_stream)
    sctx.register_pair(P[0], Q[0], pairs[0][2], pairs[0][3])

    def singles():
        out = []
        for i in range(m):
            sctx.set_params(pair_id=i)
            out.append(sctx.register_pair(P[i], Q[i], pairs[i][2], pairs[i][3]))
        return out
    single_ms, single = _timed(stream, flush, singles)
    sctx.close()
    # tensor-core matching roofline on the largest pair of the batch (stage-timed)
    big = int(np.argmax([len(p[0]) * len(p[1]) for p in pairs]))
    pctx = lsr.Context(dev, stream=stream.cuda_stream, match_precision=MATCH_MODES["bf16"])
    pctx.set_profiling(True)
    for _ in range(2):
        rb = pctx.register_pair(P[big], Q[big], pairs[big][2], pairs[big][3])
    pctx.close()
    nPb, nQb = len(pairs[big][0]), len(pairs[big][1])
    ach = 2.0 * nPb * nQb * 112 / (rb.stage_ms[3] * 1e-3) / 1e12
    peak = float(pk["bf16_tflops"])
    h2d = sum(lsr.transfer_bytes(len(p[0]), len(p[1]))[0] for p in pairs)
    d2h = sum(lsr.transfer_bytes(len(p[0]), len(p[1]))[1] for p in pairs)
    identical = all(np.array_equal(single[i].T, res[i].T) and single[i].inliers == res[i].inliers for i in range(m))
    return dict(total_ms=total_ms, e2e_ms=e2e_ms, launches=launches, npts=npts, res=res,
                clocks=clk.summary(pk.get("sm_max_mhz")), single_ms=single_ms, m=m, identical=identical,
                aligned=sum(r.status == 0 for r in res), h2d=h2d, d2h=d2h,
                roofline={"kernel": "k_match_tc", "bound": "tensor", "achieved": ach, "peak": peak,
                          "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                          "work": f"2*nP*nQ*112 flop on the largest pair ({nPb} x {nQb}); matching stage time "
                                  "(operand preparation, re-rank and exact fallback included)",
                          "peak_source": "MEASURED_PEAKS.json bf16 burst (cuBLAS)"})


def run_objective(args, rank, world, pairs):
    """Config 4: one batched forward + backward of the robust alignment objective
    over all pairs per step (RobustAlignBatch), nearest neighbours recomputed in
    the backward."""
    import torch

    import paper_1801_01572_gb300 as lsr

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    n = len(pairs)
    rng = np.random.default_rng(44 + rank)
    xis = np.concatenate([rng.normal(0, 2e-3, (n, 3)), rng.normal(0, 3e-3, (n, 3))], axis=1)
    T0s = torch.tensor(np.stack([p[4] for p in pairs]))
    eps = 0.0375
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ctx = lsr.Context(dev, stream=stream.cuda_stream)
    clouds = []
    for p in pairs:
        clouds += [torch.tensor(p[0], device="cuda", requires_grad=True),
                   torch.tensor(p[1], device="cuda", requires_grad=True)]
    xt = torch.tensor(xis, dtype=torch.float64, requires_grad=True)

    def step(cl):
        with torch.cuda.stream(stream):
            E = lsr.RobustAlignBatch.apply(xt, T0s, eps, eps * eps, ctx, *cl)
            E.sum().backward()
        return E
    for _ in range(args.warmup):
        step(clouds)
    torch.cuda.synchronize()
    pk, _ = peaks()
    times = []
    with ClockSampler(dev) as clk:
        l0 = lsr.launch_count()
        for _ in range(args.steps):
            ms, _ = _timed(stream, flush, lambda: step(clouds))
            times.append(ms)
        launches = lsr.launch_count() - l0
    total_ms = float(sum(times))
    total_ms = max_over_ranks(total_ms, world)
    # end to end: the clouds copied from pinned host memory and the gradients read back, every step
    hostP = [torch.from_numpy(p[0]).pin_memory() for p in pairs]
    hostQ = [torch.from_numpy(p[1]).pin_memory() for p in pairs]

    def e2e_step():
        cl = []
        for a, b in zip(hostP, hostQ):
            cl += [a.to("cuda", non_blocking=True).requires_grad_(), b.to("cuda", non_blocking=True).requires_grad_()]
        E = step(cl)
        grads = [c.grad.to("cpu") for c in cl]
        return E.detach().cpu(), grads
    e2e_step()
    e2e = [_timed(stream, flush, e2e_step)[0] for _ in range(max(1, args.steps // 2))]
    npts = sum(len(p[0]) + len(p[1]) for p in pairs)
    ctx.close()
    return dict(total_ms=total_ms, e2e_ms=float(sum(e2e)) / len(e2e), launches=launches, npts=npts,
                clocks=clk.summary(pk.get("sm_max_mhz")), h2d=12 * npts, d2h=12 * npts + 8 * n)


def roofline(info):
    """Roofline of the kernel that dominates the step (from the stage timers)."""
    pk, src = peaks()
    st = info["stage_ms"]
    nP, nQ, last = info["nP"], info["nQ"], info["last"]
    names = ["grids", "normals", "features", "matching", "hypotheses", "consensus", "refinement"]
    k = int(np.argmax(st[:7]))
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # FFMA TFLOP/s
    if names[k] == "matching" and info["match"] != "fp32":
        # tensor-core contraction: 2 flop per multiply-add over K = 112 (hi/lo
        # split) or 48 (plain) operand columns, for every (query, database row)
        K = 112 if info["match"] == "bf16" else 48
        flops = 2.0 * float(nP) * float(nQ) * K
        ach = flops / (st[k] * 1e-3) / 1e12
        peak = float(pk["bf16_tflops"])
        return {"kernel": "k_match_tc", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "peak_source": f"{src} bf16 burst (cuBLAS)",
                "work": f"2*nP*nQ*{K} flop (stage time incl. operand preparation, re-rank and exact fallback)"}
    if names[k] == "matching":
        # brute-force FP32 NN: per (query, candidate) pair 33 terms of one subtract and
        # one fused multiply-add (3 flop, 2 issue slots: the mix's peak is 1.5 flop per
        # lane per cycle). The exact early exit skips most terms, so the dense
        # definition's rate can exceed the pipe; executed_frac is the executed terms'
        # share of the pipe (terms counted by the profiled matcher launch).
        dense = float(nP) * float(nQ) * 33
        ach = dense * 3 / (st[k] * 1e-3) / 1e12
        peak = N_SM * FP32_LANES_PER_SM * 1.5 * sm_mhz * 1e6 / 1e12
        terms = float(info["prof"].match_terms)
        # traffic: dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch
        # (profiles/k_match_fp32_room150k_dram.md)
        traffic = 43850752 + 2816 if (nP, nQ) == (150000, 150000) else None
        return {"kernel": "k_match_fp32", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic,
                "executed_terms": terms, "executed_share": terms / dense,
                "executed_frac": terms * 3 / (st[k] * 1e-3) / 1e12 / peak,
                "note": "frac counts the dense definition's work; the exact early exits skip most terms, so it "
                        "exceeds 1 by design; executed_frac is the pipe share of the terms actually evaluated",
                "peak_source": f"152 SMs x 128 FP32 lanes x 1.5 flop x {sm_mhz:.0f} MHz (FADD+FFMA issue peak)",
                "work": "nP*nQ*33 terms x 3 flop (dense definition)"}
    if names[k] == "consensus":
        # per (hypothesis, point) query: the rigid transform (9 FMA) and the
        # squared-distance test of the points within eps (counted at one candidate)
        q = float(last.n_normal_ok) * nP
        flops = q * (18 + 8)
        ach = flops / (st[k] * 1e-3) / 1e12
        return {"kernel": "k_consensus", "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None, "queries": q,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz", "work": "queries*26 flop"}
    # other stages: report HBM against the algorithmic bytes of the stage's inputs and outputs
    bytes_ = float(nP + nQ) * (12 + 16 * 4 + 2 * 144)
    ach = bytes_ / (st[k] * 1e-3) / 1e9
    return {"kernel": names[k], "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_source": src}


# ---------------------------------------------------------------- oracle timing
def cpu_sample(fp, n_ok: int, iters: int, H: int, budget: float = 1.0):
    """Seconds the FP64 oracle needs for one pair, estimated from a bounded
    sample of every stage (normals of all points; SPFH/FPFH, descriptor NN and
    pre-rejection on fractions; consensus on a few poses; two refinement steps
    per level), each scaled to the full stage. budget scales the sample size."""
    import oracle
    rng = np.random.default_rng(0)
    P, Q = fp.P.astype(np.float64), fp.Q.astype(np.float64)
    nP, nQ = len(P), len(Q)
    t_total, parts = 0.0, {}

    def tm(fn):
        t0 = time.perf_counter()
        out = fn()
        return time.perf_counter() - t0, out

    dt, (NP, _, _, _) = tm(lambda: oracle.normals(P, fp.vpP, 0.05))
    parts["normals"] = dt * (nP + nQ) / nP
    m = max(64, int(0.02 * budget * nP))
    qi = np.sort(rng.choice(nP, m, replace=False))
    dt, _ = tm(lambda: oracle.spfh(P, NP, 0.125, qidx=qi))
    parts["spfh"] = dt * (nP + nQ) / m
    dt, _ = tm(lambda: oracle.fpfh(P, NP, np.zeros((nP, 33)), 0.125, qidx=qi))
    parts["fpfh"] = dt * (nP + nQ) / m
    F = rng.uniform(size=(nP, 33))
    mq = max(16, int(100 * budget))
    dt, _ = tm(lambda: oracle.match(F, F[:nQ] if nQ <= nP else rng.uniform(size=(nQ, 33)),
                                    qidx=rng.choice(nP, mq, replace=False)))
    parts["matching"] = dt * nP / mq
    hs = max(10_000, int(200_000 * budget))
    nn = rng.integers(0, nQ, nP)
    v = np.ones(max(nP, nQ), np.uint8)
    dt, _ = tm(lambda: oracle.hypotheses(P, Q, nn, v[:nP], v[:nQ], hs, 1, 0, 0.9))
    parts["hypotheses"] = dt * H / hs
    npose = max(8, int(8 * budget))
    from synth import random_pose
    Rs, ts = [], []
    for i in range(npose):
        # most tested hypotheses are wrong; one pose in eight is the true one
        T = fp.T if i % 8 == 0 else random_pose(rng) @ fp.T
        Rs.append(T[:3, :3])
        ts.append(T[:3, 3])
    dt, _ = tm(lambda: oracle.consensus(P, Q, np.array(Rs), np.array(ts), 0.0375))
    parts["consensus"] = dt * max(n_ok, 1) / npose
    dt, _ = tm(lambda: oracle.refine(P, Q, fp.T, 0.0375, 0.0375 ** 2, iters=2, tol=0.0))
    parts["refinement"] = dt / 2 * max(iters, 1)
    t_total = sum(parts.values())
    return t_total, parts


def cpu_baseline_line(fp, n_ok, iters, H, budget=1.0):
    import oracle
    secs, parts = cpu_sample(fp, n_ok, iters, H, budget)
    return {"value": 1.0 / secs, "unit": "pairs/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": ("FP64 C oracle (pthreads): normals of all points; SPFH/FPFH of %.0f%% of the points; "
                       "descriptor NN of %d queries; pre-rejection of %d hypotheses; consensus of %d poses; "
                       "2 refinement steps; each scaled to the full pair (%d normal-checked hypotheses, "
                       "%d refinement steps as the GPU run)") % (2 * budget, max(16, int(100 * budget)),
                                                               max(10_000, int(200_000 * budget)),
                                                               max(8, int(8 * budget)), n_ok, iters),
            "stage_s": {k: round(v, 3) for k, v in parts.items()}}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle on bounded samples of the workload, one sample per step."""
    if rank != 0:
        return None
    import oracle
    from synth import make_pair
    oracle.build()
    fp = make_pair(args.config, pair=0)
    n_ok = {0: 6900, 1: 8700}.get(args.config, 8000)  # normal-checked hypotheses of the workload
    iters = 120
    H = 4_000_000
    budget = 2.0
    for _ in range(args.warmup):
        cpu_sample(fp, n_ok, iters, H, budget=0.25)
    secs = []
    for _ in range(args.steps):
        s, parts = cpu_sample(fp, n_ok, iters, H, budget=budget)
        secs.append(s)
    value = len(secs) / sum(secs)
    cores = oracle.threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": "per step: normals of all points, 4% of SPFH/FPFH, 200 descriptor-NN "
                                       "queries, 400k hypotheses, 16 consensus poses (1 in 8 the true one), "
                                       "2 refinement steps, each scaled to the full pair"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=1, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--match", default="fp32", choices=sorted(MATCH_MODES))
    ap.add_argument("--points", type=int, default=None,
                    help="points per cloud instead of the configuration's (a smaller case of the same scene, "
                         "for profiler captures)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="do not also time the other descriptor matchers")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    pairs = batch_pairs(args.config, rank) if args.config in BATCH_PAIRS and args.impl == "ours" else None
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    if args.config == 4:
        info = run_objective(args, rank, world, pairs)
        if rank == 0:
            K, n = args.steps, len(pairs)
            value = job_rate(K * n, world, info["total_ms"])
            line = {
                "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": info["total_ms"] / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS[4], "pairs_per_step": n, "points_per_step": info["npts"],
                           "l2": "flushed between steps by a 256 MB write outside the timed events",
                           "parallelism": "replicas (one batch per GPU)" if world > 1 else "single GPU"},
                "points_per_s": value * info["npts"] / n,
                "e2e": {"value": world * n / (info["e2e_ms"] * 1e-3), "unit": "pairs/s",
                        "h2d_bytes_per_step": info["h2d"] * world, "d2h_bytes_per_step": info["d2h"] * world},
                "gpu_launches": int(info["launches"]), "clocks": info["clocks"],
            }
            # algorithmic bytes: the forward and the backward each read both clouds once,
            # the backward writes dP and dQ (12 B per point each way)
            pk, src = peaks()
            ach = 36.0 * info["npts"] / (line["ms_per_step"] * 1e-3) / 1e9
            line["roofline"] = {"kernel": "objective fwd+bwd (whole step)", "bound": "hbm", "achieved": ach,
                                "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": None,
                                "work": "36 B per point per step over the step time", "peak_source": src}
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    if args.config in (2, 3):
        info = run_batch(args, rank, world, pairs)
        N_BATCH = len(pairs)
        if rank == 0:
            K = args.steps
            value = job_rate(K * N_BATCH, world, info["total_ms"])
            line = {
                "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": info["total_ms"] / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config], "pairs_per_step": N_BATCH,
                           "points_per_step": info["npts"],
                           "l2": "flushed between steps by a 256 MB write outside the timed events",
                           "parallelism": "replicas (one batch per GPU)" if world > 1 else "single GPU"},
                "points_per_s": value * info["npts"] / N_BATCH,
                "result": {"aligned": info["aligned"]},
                "roofline": info["roofline"],
                "e2e": {"value": world * N_BATCH / (info["e2e_ms"] * 1e-3), "unit": "pairs/s",
                        "h2d_bytes_per_step": info["h2d"] * world, "d2h_bytes_per_step": info["d2h"] * world},
                "gpu_launches": int(info["launches"]),
                "variants": {"fp32_single_pair": {
                    "value": info["m"] / (info["single_ms"] * 1e-3), "unit": "pairs/s",
                    "sample": f"first {info['m']} of the {N_BATCH} pairs, lsr_register_pair one after another, "
                              "FP32 matching",
                    "identical_pose": info["identical"]}},
                "clocks": info["clocks"],
            }
            if args.config == 3:
                # pose error against the FP64 oracle on two pairs: the oracle's graduated
                # refinement from the generator's pose reaches the fixed point the path converges to
                import oracle
                from synth import pose_error
                errs = []
                for i in (0, 1):
                    T_ref, _ = oracle.refine_gnc(pairs[i][0], pairs[i][1], pairs[i][4], 0.0375, 1.0, levels=3, iters=50)
                    errs.append(pose_error(info["res"][i].T, T_ref))
                line["result"]["oracle_pose_error"] = {"deg": max(e[0] for e in errs), "m": max(e[1] for e in errs),
                                                       "pairs": 2}
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    info = run_ours(args, rank, world)
    if rank == 0:
        K = args.steps
        value = job_rate(K, world, info["total_ms"])
        e2e = job_rate(K, world, info["e2e_ms"])
        last = info["last"]
        prm = info["params"]
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": info["total_ms"] / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config] if args.points is None else
                       f"{WORKLOADS[args.config]}, resized to {args.points} points per cloud",
                       "points": [info["nP"], info["nQ"]],
                       "hypotheses": int(prm.n_hypotheses), "match": args.match, "refine_levels": int(prm.refine_levels),
                       "l2": "flushed between steps by a 256 MB write outside the timed events",
                       "parallelism": "replicas (one pair per GPU)" if world > 1 else "single GPU"},
            "points_per_s": value * (info["nP"] + info["nQ"]),
            "stage_ms": {n: round(float(v), 3) for n, v in zip(
                ["grids", "normals", "features", "matching", "hypotheses", "consensus", "refinement", "total"],
                info["stage_ms"])},
            "result": {"inliers": last.inliers, "survivors": last.survivors, "normal_ok": last.n_normal_ok,
                       "refine_iters": last.refine_iters, "match_fallbacks": last.match_fallbacks},
            "roofline": roofline(info),
            "information_matrix": info["information"],
            "surfel_correction": info["surfels"],
            "voxel_downsample": info["voxel"],
            "e2e": {"value": e2e, "unit": "pairs/s", "h2d_bytes_per_step": info["h2d"] * world,
                    "d2h_bytes_per_step": info["d2h"] * world},
            "gpu_launches": int(info["launches"]),
            "variants": info["variants"],
            "clocks": info["clocks"],
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_line(info["fp"], last.n_normal_ok, last.refine_iters,
                                                     int(prm.n_hypotheses), budget=12.0)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
