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
    # the dominant kernel is bracketed by two CUDA events on the context stream
    # in every timed step (its only added work: two event records per step)
    main_kernel = "k_match_win" if args.match == "fp32" else "k_match_tc"
    ctx.set_kernel_timing(main_kernel)
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
    main_times = ctx.kernel_times()
    ctx.set_kernel_timing(None)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = float(sum(times))
    total_ms = max_over_ranks(total_ms, world)
    # per-stage device times (and the FP32 matcher's term count) from profiled
    # runs after the timed region: stage events and the counting matcher
    ctx.set_profiling(True)
    ctx.set_kernel_timing("")
    n_prof = min(args.steps, 3)
    for _ in range(n_prof):
        with torch.cuda.stream(stream):
            flush.zero_()
        prof = ctx.register_pair(P, Q, fp.vpP, fp.vpQ)
        stages += np.array(prof.stage_ms)
    ctx.set_profiling(False)
    kernel_times = ctx.kernel_times()
    ctx.set_kernel_timing(None)
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
                main_kernel=main_kernel, main_times=main_times, kernel_times=kernel_times, n_prof=n_prof,
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

    # the consensus variants (single-cell lookup, per-inlier normal check) on this
    # pair and on the 5k-point objects pair
    info["speed_modes"] = None
    if world == 1 and args.variants:
        from synth import make_pair as _mk
        fp0 = _mk(0, 0)
        P0, Q0 = torch.from_numpy(fp0.P).cuda(), torch.from_numpy(fp0.Q).cuda()
        with lsr.Context(dev, stream=stream.cuda_stream) as c0:
            base0 = c0.register_pair(P0, Q0, fp0.vpP, fp0.vpQ)
        info["speed_modes"] = {"this_pair": speed_modes(dev, stream, flush, fp, P, Q, last),
                               "objects_5k": speed_modes(dev, stream, flush, fp0, P0, Q0, base0)}
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
            vkern = "k_match_win" if name == "fp32" else "k_match_tc"
            vctx.set_kernel_timing(vkern)
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
            vtimes = vctx.kernel_times()
            vctx.close()
            info["variants"][name] = {
                "value": args.steps / (sum(vt) * 1e-3), "unit": "pairs/s", "ms_per_step": sum(vt) / args.steps,
                "match_ms": float(vst[3] / args.steps), "match_fallbacks": vl.match_fallbacks,
                "identical_pose": bool(np.array_equal(vl.T, last.T)) and vl.inliers == last.inliers,
                "kernel_times": vtimes}
    return info


# ---------------------------------------------------------------- oracle poses
GOLDEN = os.path.join(ROOT, "tests", "golden", "registrations.json")


def golden_entries():
    """Complete FP64 oracle registrations stored by tests/golden/make_registrations.py."""
    try:
        with open(GOLDEN) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def golden_error(config: int, pair: int, pair_id: int, T):
    """(deg, m) between a pose and the oracle's registration of the same pair
    and RNG key, or None if that registration is not stored."""
    from synth import pose_error
    e = golden_entries().get(f"c{config}_p{pair}_k{pair_id}")
    if e is None:
        return None
    ang, tr = pose_error(np.asarray(T), np.array(e["T"]).reshape(4, 4))
    return {"deg": ang, "mm": tr * 1e3, "within_0.05deg_0.5mm": bool(ang < 0.05 and tr < 5e-4)}


# ---------------------------------------------------------------- variant modes
def speed_modes(dev, stream, flush, fp, P, Q, base, steps=3):
    """The consensus variants against the exact default on one pair: the
    single-cell lookup of eq. (1) (the paper's speed argument) and the
    per-inlier normal check. Per mode: pairs/s and consensus-stage ms (stage
    events), the selected hypothesis' count and pose against the exact mode's,
    the refined pose against it; for the single cell also its recall: the
    share of the exact search's inliers at the exact mode's refined pose that
    the own-cell lookup still finds within eps."""
    import paper_1801_01572_gb300 as lsr
    from synth import pose_error
    out = {}
    eps = 0.0375
    ctx0 = lsr.Context(dev, stream=stream.cuda_stream)
    ctx0.set_profiling(True)
    ref = ctx0.register_pair(P, Q, fp.vpP, fp.vpQ)
    T = np.asarray(base.T)
    X = (fp.P.astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)
    _, de = ctx0.stage_nn(Q, X, eps, lsr.NN_EXACT)
    _, ds = ctx0.stage_nn(Q, X, eps, lsr.NN_SINGLE_CELL)
    n_exact = int((de < eps * eps).sum())
    n_single = int((ds < eps * eps).sum())
    ctx0.close()
    for name, kw in (("exact", {}), ("single_cell", {"nn_mode": lsr.NN_SINGLE_CELL}),
                     ("inlier_normals", {"normal_mode": lsr.NORMALS_INLIERS})):
        c = lsr.Context(dev, stream=stream.cuda_stream, **kw)
        c.set_profiling(True)
        c.register_pair(P, Q, fp.vpP, fp.vpQ)
        ts, cons, r = [], [], None
        for _ in range(steps):
            ms, r = _timed(stream, flush, lambda: c.register_pair(P, Q, fp.vpP, fp.vpQ))
            ts.append(ms)
            cons.append(r.stage_ms[5])
        c.close()
        ah, th = pose_error(r.T_hyp, ref.T_hyp)
        af, tf = pose_error(r.T, ref.T)
        out[name] = {"pairs_per_s": steps / (sum(ts) * 1e-3), "consensus_ms": float(np.mean(cons)),
                     "hypotheses_tested": int(r.n_normal_ok), "selected_h": int(r.best_h),
                     "selected_inliers": int(r.hyp_inliers),
                     "hypothesis_pose_vs_exact": {"deg": ah, "mm": th * 1e3},
                     "refined_pose_vs_exact": {"deg": af, "mm": tf * 1e3},
                     "inliers": int(r.inliers)}
    out["single_cell"]["recall_at_refined_pose"] = n_single / max(n_exact, 1)
    out["single_cell"]["inliers_exact_vs_single"] = [n_exact, n_single]
    out["note"] = ("stage times with stage events on; the refinement stays exact in every mode, so a variant changes "
                   "only which hypothesis seeds it")
    return out


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


def run_headline(dev, pairs, steps=2):
    """The headline comparison on config 2's 256 uneven room pairs: the batched
    tensor-core path (one lsr_register_batch per step: BF16 matching with FP32
    re-rank, concurrent streams, one CUDA graph, autotuned tiles) against the
    plain FP32 path registering the same pairs one lsr_register_pair after
    another, both timed with CUDA events on resident inputs in this run. Parity:
    the two paths' poses must be identical, and the poses of the pairs that have
    a stored FP64 oracle registration are compared with it."""
    import torch

    import paper_1801_01572_gb300 as lsr
    P = [torch.from_numpy(p[0]).cuda() for p in pairs]
    Q = [torch.from_numpy(p[1]).cuda() for p in pairs]
    vp = np.concatenate([np.concatenate([p[2], p[3]]) for p in pairs]).astype(np.float32)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    bctx = lsr.Context(dev, stream=stream.cuda_stream, match_precision=MATCH_MODES["bf16"], batch_graph=1)
    for _ in range(3):  # tunes tiles and streams, captures the graph, replays once
        bctx.register_batch(P, Q, vp)
    bt = []
    for _ in range(steps):
        ms, res = _timed(stream, flush, lambda: bctx.register_batch(P, Q, vp))
        bt.append(ms)
    bctx.close()
    sctx = lsr.Context(dev, stream=stream.cuda_stream)
    sctx.register_pair(P[0], Q[0], pairs[0][2], pairs[0][3])

    def singles():
        out = []
        for i in range(len(pairs)):
            sctx.set_params(pair_id=i)
            out.append(sctx.register_pair(P[i], Q[i], pairs[i][2], pairs[i][3]))
        return out
    single_ms, single = _timed(stream, flush, singles)
    sctx.close()
    n = len(pairs)
    identical = all(np.array_equal(single[i].T, res[i].T) and single[i].inliers == res[i].inliers for i in range(n))
    errs = {}
    for i in range(n):
        g = golden_error(2, i, i, res[i].T)
        if g is not None:
            errs[f"pair {i} ({len(pairs[i][0])} + {len(pairs[i][1])} points)"] = g
    batched = n * steps / (sum(bt) * 1e-3)
    single_rate = n / (single_ms * 1e-3)
    return {"workload": WORKLOADS[2], "pairs": n, "points": int(sum(len(p[0]) + len(p[1]) for p in pairs)),
            "batched_bf16": {"value": batched, "unit": "pairs/s", "ms_per_batch": sum(bt) / steps, "steps": steps},
            "fp32_single_pair": {"value": single_rate, "unit": "pairs/s", "ms_all_pairs": single_ms},
            "speedup": batched / single_rate,
            "identical_poses_all_pairs": bool(identical),
            "aligned": int(sum(r.status == 0 for r in res)),
            "oracle_pose_error": {"pairs_compared": len(errs),
                                  "max_deg": max((e["deg"] for e in errs.values()), default=None),
                                  "max_mm": max((e["mm"] for e in errs.values()), default=None),
                                  "all_within_0.05deg_0.5mm": all(e["within_0.05deg_0.5mm"] for e in errs.values())
                                  if errs else None,
                                  "per_pair": errs,
                                  "reference": "complete FP64 oracle registrations of the same pairs and RNG keys "
                                               "(tests/golden/registrations.json)"},
            "l2": "flushed before each timed call by a 256 MB write outside the timed events"}


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


def _kernel_avg_ms(times: dict, prefix: str):
    """(launches, average ms) of the timed kernels whose name starts with prefix."""
    n = sum(v[0] for k, v in times.items() if k.startswith(prefix))
    ms = sum(v[1] for k, v in times.items() if k.startswith(prefix))
    return n, (ms / n if n else None)


def fp32_alu_peak(sm_mhz: float) -> float:
    """Issue peak of the matcher's instruction mix, TFLOP/s: one FADD and one
    FFMA per term (3 flop in 2 issue slots, 1.5 flop per lane per cycle)."""
    return N_SM * FP32_LANES_PER_SM * 1.5 * sm_mhz * 1e6 / 1e12


def roofline(info):
    """Roofline of the kernel that dominates the step, from its CUDA-event
    durations in the timed steps (events on the context stream around each of
    its launches)."""
    pk, src = peaks()
    nP, nQ = info["nP"], info["nQ"]
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    n, avg = _kernel_avg_ms(info["main_times"], info["main_kernel"])
    if info["main_kernel"] == "k_match_tc":
        K = 112 if info["match"] == "bf16" else 48
        flops = 2.0 * float(nP) * float(nQ) * K
        ach = flops / (avg * 1e-3) / 1e12
        peak = float(pk["bf16_tflops"])
        return {"kernel": "k_match_tc", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "launch_ms": avg, "launches_timed": n,
                "peak_source": f"{src} bf16 burst (cuBLAS), of measured",
                "work": f"2*nP*nQ*{K} flop per launch (the contraction the kernel executes)"}
    # FP32 matcher: the terms it evaluates (counted by the profiled launch; the
    # count does not depend on timing), one subtract and one fused multiply-add
    # each, against the issue peak of that mix
    terms = float(info["prof"].match_terms)
    dense = float(nP) * float(nQ) * 33
    peak = fp32_alu_peak(sm_mhz)
    ach = terms * 3 / (avg * 1e-3) / 1e12
    # traffic: dram__bytes_read.sum + dram__bytes_write.sum of one full-size
    # launch of this kernel on the room pair, from an ncu capture (the two
    # descriptor tables read once; the tiles' rows re-read from L2)
    traffic = 47619328 + 600832 if (nP, nQ) == (150000, 150000) else None
    return {"kernel": "k_match_win", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": traffic, "launch_ms": avg, "launches_timed": n,
            "algorithmic_bytes": 144.0 * (nP + nQ) + 8.0 * nP,
            "executed_terms": terms, "executed_share": terms / dense,
            "dense_equivalent": {"achieved": dense * 3 / (avg * 1e-3) / 1e12, "unit": "TFLOP/s",
                                 "note": "rate of the definition's nP*nQ*33 terms; the projection window and the "
                                         "exact early exits skip "
                                         f"{100 * (1 - terms / dense):.1f}% of them, so it is no roofline fraction"},
            "peak_source": f"152 SMs x 128 FP32 lanes x 1.5 flop x {sm_mhz:.0f} MHz (FADD+FFMA issue peak)",
            "work": "executed terms x 3 flop (subtract + fused multiply-add), terms counted by the profiled launch"}


def roofline_tc(info):
    """Tensor-pipe roofline of the BF16 matcher from the bf16 variant's timed
    steps: the contraction at the configuration's padded K = 48 and at the
    K = 112 the hi/lo operand split executes, against the measured BF16 peak."""
    v = info.get("variants", {}).get("bf16")
    if not v or "kernel_times" not in v:
        return None
    pk, src = peaks()
    n, avg = _kernel_avg_ms(v["kernel_times"], "k_match_tc")
    if not avg:
        return None
    nP, nQ = float(info["nP"]), float(info["nQ"])
    peak = float(pk["bf16_tflops"])
    a48 = 2 * nP * nQ * 48 / (avg * 1e-3) / 1e12
    a112 = 2 * nP * nQ * 112 / (avg * 1e-3) / 1e12
    return {"kernel": "k_match_tc", "bound": "tensor", "launch_ms": avg, "launches_timed": n, "peak": peak,
            "unit": "TFLOP/s", "peak_source": f"{src} bf16 burst (cuBLAS), of measured",
            "padded_k48": {"achieved": a48, "frac": a48 / peak, "work": "2*nP*nQ*48 flop (the configuration's "
                                                                        "descriptors zero-padded to 48)"},
            "executed_k112": {"achieved": a112, "frac": a112 / peak, "work": "2*nP*nQ*112 flop (hi/lo BF16 split "
                                                                            "the kernel executes)"},
            "match_fallbacks": v.get("match_fallbacks"), "traffic": None}


# Algorithmic HBM bytes (or flops) of one registration step per kernel family,
# from the arrays each kernel reads and writes once (the work column of the
# kernel table in the design notes); both clouds together.
def _kernel_work(name, nP, nQ, res, prm, terms):
    N = nP + nQ
    S, n_ok, H = res.survivors, res.n_normal_ok, int(prm.n_hypotheses)
    table = [
        ("k_match_win", "alu", 3.0 * terms, "flop", "executed terms x 3 flop"),
        ("k_match_tc", "tensor", 2.0 * nP * nQ * 112, "flop", "2*nP*nQ*112 flop"),
        ("k_normals", "hbm", 48.0 * N, "B", "16 B point + 16 B grid copy in, 16 B normal out"),
        ("k_spfh", "hbm", 176.0 * N, "B", "16 B point + 16 B normal in, 144 B SPFH row out"),
        ("k_fpfh", "hbm", 320.0 * N, "B", "16 B point + 16 B normal + 144 B SPFH row in, 144 B FPFH row out"),
        ("k_proj", "hbm", 152.0 * N, "B", "144 B FPFH row in, 8 B projection and bound out"),
        ("k_gather_db", "hbm", 300.0 * nQ, "B", "4 B order + 8 B projection + 144 B row in, 144 B row out "
                                                "(Q: the database)"),
        ("k_prep_tiles", "hbm", (144.0 + 224.0) * N, "B", "144 B FPFH row in, 224 B BF16 operand row out"),
        ("k_hyp_count", "hbm", 36.0 * N, "B", "unique bytes of the sampled arrays (points, normals, nn)"),
        ("k_hyp_gather", "hbm", 8.0 * S, "B", "4 B per survivor id in, 4 B out"),
        ("k_rigid_survivors", "hbm", 321.0 * S, "B", "per survivor 4 x (P, Q points and normals, nn) in, 49 B out"),
        ("k_consensus_count<true>", "hbm", 16.0 * nP + 56.0 * n_ok, "B",
         "16 B per P point, 56 B per normal-checked pose (L1/L2-resident table lookups dominate)"),
        ("k_pack", "hbm", 28.0 * N, "B", "12 B xyz in, 16 B float4 out"),
        ("k_bbox_partial", "hbm", 12.0 * N, "B", "12 B xyz in"),
    ]
    for pre, bound, work, unit, what in table:
        if name.startswith(pre):
            return bound, work, unit, what
    return None


def kernel_table(info):
    """Every kernel of the profiled steps: launches per step, average duration,
    share of the summed kernel time, and, where the work is defined, the
    achieved rate against the relevant peak."""
    pk, src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    steps = info["n_prof"]
    kt = info["kernel_times"]
    tot = sum(v[1] for v in kt.values()) or 1.0
    rows = []
    for name, (n, ms) in sorted(kt.items(), key=lambda x: -x[1][1]):
        row = {"kernel": name, "launches_per_step": n / steps, "avg_us": 1e3 * ms / n, "share": ms / tot}
        w = _kernel_work(name, info["nP"], info["nQ"], info["prof"], info["params"],
                         float(info["prof"].match_terms))
        if w is not None:
            bound, work, unit, what = w
            per_step_s = ms / steps * 1e-3
            if unit == "B":
                ach = work / per_step_s / 1e9
                row.update(bound=bound, work_per_step=work, achieved=ach, unit="GB/s", peak=pk["hbm_gbs"],
                           frac=ach / pk["hbm_gbs"], work=what)
            else:
                ach = work / per_step_s / 1e12
                peak = fp32_alu_peak(sm_mhz) if bound == "alu" else float(pk["bf16_tflops"])
                row.update(bound=bound, work_per_step=work, achieved=ach, unit="TFLOP/s", peak=peak,
                           frac=ach / peak, work=what)
        rows.append(row)
    return {"source": f"CUDA events around every launch of {steps} profiled registrations after the timed steps "
                      "(same resident inputs); shares are of the summed kernel time",
            "peak_source": f"{src} (HBM, BF16); FP32 issue peak derived from 152 SMs x 128 lanes x {sm_mhz:.0f} MHz",
            "kernels": rows}


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


CPU_SAMPLE = ("FP64 C oracle (pthreads): normals of all points; SPFH/FPFH of {pct:.0f}% of the points; descriptor "
              "NN of {mq} queries; pre-rejection of {hs} hypotheses; consensus of {npose} poses (1 in 8 the true one); "
              "2 refinement steps; each stage's time scaled by full size / sample size ({n_ok} normal-checked "
              "hypotheses, {iters} refinement steps) and summed")


def _sample_text(budget, n_ok, iters):
    return CPU_SAMPLE.format(pct=2 * budget, mq=max(16, int(100 * budget)), hs=max(10_000, int(200_000 * budget)),
                             npose=max(8, int(8 * budget)), n_ok=n_ok, iters=iters)


def oracle_full_config0():
    """Seconds of one complete oracle registration of the config-0 pair (5k + 5k
    points): measured, not extrapolated."""
    import oracle
    from synth import make_pair
    fp = make_pair(0, 0)
    t0 = time.perf_counter()
    r = oracle.register(fp.P, fp.Q, fp.vpP, fp.vpQ, seed=0)
    return time.perf_counter() - t0, r


def cpu_baseline_line(fp, n_ok, iters, H, budget=4.0, config=1):
    """The oracle on the host cores: the stage-sampled estimate for this
    workload (the same sampling as --impl reference), and one complete
    registration of the config-0 pair, measured."""
    import oracle
    oracle.build()
    if config == 0:
        secs, _ = oracle_full_config0()
        return {"value": 1.0 / secs, "unit": "pairs/s", "cores": oracle.threads(), "kind": "oracle",
                "estimate": False, "sample": "one complete FP64 oracle registration of the pair (5k + 5k points)"}
    secs, parts = cpu_sample(fp, n_ok, iters, H, budget)
    c0, _ = oracle_full_config0()
    return {"value": 1.0 / secs, "unit": "pairs/s", "cores": oracle.threads(), "kind": "oracle", "estimate": True,
            "sample": _sample_text(budget, n_ok, iters), "formula": "1 / sum over stages (sample s x full / sample)",
            "stage_s": {k: round(v, 3) for k, v in parts.items()},
            "measured_config0": {"workload": WORKLOADS[0], "value": 1.0 / c0, "unit": "pairs/s", "seconds": c0,
                                 "sample": "one complete FP64 oracle registration (not extrapolated)"}}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle on the host cores, one bounded sample of the workload per
    step. On config 0 a step is one complete registration (measured); on the
    larger configurations a step is the stage sample of cpu_sample, and its
    value is the fraction of a pair the sample stands for over the step's wall
    time (so steps x ms_per_step is the real duration of the run)."""
    if rank != 0:
        return None
    import oracle
    from synth import make_pair
    oracle.build()
    fp = make_pair(args.config, pair=0)
    n_ok = {0: 6900, 1: 8700}.get(args.config, 8000)  # normal-checked hypotheses of the workload
    iters = 120
    H = 4_000_000
    budget = 4.0
    full = args.config == 0
    for _ in range(args.warmup):
        if not full:
            cpu_sample(fp, n_ok, iters, H, budget=0.25)
    walls, frac = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        if full:
            oracle_full_config0()
            frac.append(1.0)
        else:
            est, _ = cpu_sample(fp, n_ok, iters, H, budget=budget)
            frac.append((time.perf_counter() - t0) / est)
        walls.append(time.perf_counter() - t0)
    value = sum(frac) / sum(walls)
    cores = oracle.threads()
    sample = "one complete FP64 oracle registration per step" if full else _sample_text(budget, n_ok, iters)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "parallelism": "host threads"},
            "pair_fraction_per_step": sum(frac) / len(frac),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "estimate": not full},
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
    ap.add_argument("--no-headline", dest="headline", action="store_false",
                    help="do not also time the batched BF16 path against the FP32 single-pair path on config 2")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    pairs = batch_pairs(args.config, rank) if args.config in BATCH_PAIRS and args.impl == "ours" else None
    # the headline's 256 pairs are generated by host processes spawned before
    # any GPU work
    head_pool = head_async = None
    if args.impl == "ours" and args.config in (0, 1) and args.headline and world == 1 and args.points is None:
        import multiprocessing as mp
        head_pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
        head_async = head_pool.map_async(_gen_pair, [(2, i) for i in rank_pair_ids(2, 0)], chunksize=2)
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
            # pose error against complete FP64 oracle registrations of the pairs that have one
            errs = {}
            for i in range(N_BATCH):
                g = golden_error(args.config, i, i, info["res"][i].T)
                if g is not None:
                    errs[f"pair {i}"] = g
            line["result"]["oracle_pose_error"] = {
                "pairs_compared": len(errs), "max_deg": max((e["deg"] for e in errs.values()), default=None),
                "max_mm": max((e["mm"] for e in errs.values()), default=None),
                "all_within_0.05deg_0.5mm": all(e["within_0.05deg_0.5mm"] for e in errs.values()) if errs else None,
                "reference": "complete FP64 oracle registrations (tests/golden/registrations.json)"}
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    # the generator processes finish before any timed region: running beside
    # it, they would take the host cores the launching thread needs
    head_pairs = None
    if head_async is not None:
        head_pairs = head_async.get()
        head_pool.close()
        head_pool.join()
    info = run_ours(args, rank, world)
    headline = None
    if head_pairs is not None:
        headline = run_headline(int(os.environ.get("LOCAL_RANK", 0)), head_pairs)
        del head_pairs
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
                       "refine_iters": last.refine_iters, "match_fallbacks": last.match_fallbacks,
                       "oracle_pose_error": golden_error(args.config, rank, 0, last.T) if args.points is None
                       else None},
            "roofline": roofline(info),
            "roofline_tc": roofline_tc(info),
            "kernels": kernel_table(info),
            "information_matrix": info["information"],
            "surfel_correction": info["surfels"],
            "voxel_downsample": info["voxel"],
            "e2e": {"value": e2e, "unit": "pairs/s", "h2d_bytes_per_step": info["h2d"] * world,
                    "d2h_bytes_per_step": info["d2h"] * world},
            "gpu_launches": int(info["launches"]),
            "variants": info["variants"],
            "speed_modes": info["speed_modes"],
            "clocks": info["clocks"],
        }
        if headline is not None:
            line["headline"] = headline
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_line(info["fp"], last.n_normal_ok, last.refine_iters,
                                                     int(prm.n_hypotheses), budget=4.0, config=args.config)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
