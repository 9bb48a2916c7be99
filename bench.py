#!/usr/bin/env python
"""Benchmark of the Flow Fields dense-matching stage (FlowFields++, arXiv 1805.03517, Sec. 3.1) on GB300.

One step = the whole stage for one frame pair: features (pyramid + Walsh-Hadamard descriptors) of both frames,
exact initial matches, per-level propagation with random search in both directions, and the forward/backward
consistency check.  Metric: Mpx/s = level-0 pixels of frame 1 matched per second (bidirectional).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (the path has no exchange between pairs; weak
scaling); rank 0 prints one JSON line with the max-over-ranks step time.  ``--impl reference`` times the CPU
oracle (the reference arm of this benchmark) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpx/s bidirectional FF matching, batched/served vs single-pair; p50/p99 latency"
UNIT = "Mpx/s"
L2_FLUSH_BYTES = 512 << 20
ALG_BYTES_PER_PIXEL_ITER = 11 * 96 + 96 + 8  # candidate gathers + own descriptor + flow/cost, per direction
ALG_BYTES_PER_PIXEL_ITER_CENSUS = 11 * 32 + 32 + 8  # the same with 32-byte Census patterns
COSTS = {"wht_sad": 0, "census": 1}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="kitti_1242x375")
    ap.add_argument("--cost", default="wht_sad", choices=["wht_sad", "census"],
                    help="matching cost of the timed workload (Census: 7x7 patterns, Hamming distance)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-pair batched measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream measurement")
    ap.add_argument("--no-census", action="store_true", help="skip the Census-cost measurement")
    ap.add_argument("--no-sub-scales", action="store_true", help="skip the measurement with sub-scale grids")
    ap.add_argument("--settle-s", type=float, default=2.0,
                    help="seconds of untimed steps before the warm-up steps, so the clocks have settled")
    ap.add_argument("--no-filtered", action="store_true",
                    help="skip the measurement with two consistency checks and sparsification")
    ap.add_argument("--autotune", action="store_true",
                    help="run the autotuner instead of the package's table of tuned configurations")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--features", default="frames", choices=["frame", "batch", "frames"],
                    help="features of the step's frames: one ff_features call per frame, ff_features_batch, or "
                         "ff_match_frames (features and matching in one call, the fine levels' descriptors beside "
                         "the coarse levels' matching)")
    ap.add_argument("--overlap", type=int, default=2, choices=[0, 1, 2],
                    help="with --features frames: where the fine levels' descriptors fork off (FF_OPT_OVERLAP)")
    ap.add_argument("--tuning", default=None,
                    help="JSON list of per-level [tile_w, tile_h, iters_per_launch, threads, speculate] instead of "
                         "autotuning (for reproducible profiler captures)")
    return ap.parse_args()


def aggregate_ranks(torch, dist, dev, ms_local, px_per_step, world):
    """Weak scaling over replicas: the slowest rank's step time, and the pixels all ranks matched per second.
    Returns (ms_per_step over ranks, Mpx/s of the whole job)."""
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, px_per_step * world / (ms / 1000.0) / 1e6


def prop_kernel(cfg):
    """The propagation kernel a level's configuration [tile w, tile h, iterations/launch, threads, speculate,
    cluster, dataflow] launches: the dataflow form, the cluster form or the tile form."""
    cfg = list(cfg)
    if len(cfg) > 6 and cfg[6]:
        return "k_propagate_df"
    if len(cfg) > 5 and cfg[5]:
        return "k_propagate_cl"
    return "k_propagate"


def propagate_l1_record(tuning):
    """The committed ncu capture of a level-0 propagation launch of the 1242x375 pair (L1 LSU data-pipe wavefronts,
    their peak per cycle, DRAM bytes), if the kernel source and the launch configuration are the ones it was
    captured with."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "propagate_l1_kitti_1242x375.json")
    src = os.path.join(ROOT, "paper_1805_03517_gb300", "csrc", "propagate.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    with open(src, "rb") as f:
        if rec.get("propagate_cu_sha256") != hashlib.sha256(f.read()).hexdigest():
            return None
    if [list(c) for c in rec.get("tiles_per_level", [])] != [list(c) for c in tuning]:
        return None
    return rec


def propagate_traffic(tuning):
    """DRAM bytes per k_propagate launch from the committed ncu capture, if the kernel source and the per-level
    launch configuration are the ones it was captured with."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "propagate_traffic_kitti_1242x375.json")
    src = os.path.join(ROOT, "paper_1805_03517_gb300", "csrc", "propagate.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if rec.get("propagate_cu_sha256") != sha:
        return None
    if [list(c) for c in rec.get("tiles_per_level", [])] != [list(c) for c in tuning]:
        return None
    return rec["dram_bytes_per_launch"]


def batch_traffic():
    """DRAM bytes per algorithmic byte of k_propagate in a batch whose features exceed L2, from the committed ncu
    capture of an 8-pair KITTI batch, if the kernel source is the one it was captured with."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "propagate_traffic_batch8_kitti_1242x375.json")
    src = os.path.join(ROOT, "paper_1805_03517_gb300", "csrc", "propagate.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    with open(src, "rb") as f:
        if rec.get("propagate_cu_sha256") != hashlib.sha256(f.read()).hexdigest():
            return None
    return rec


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled in the background during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank].strip() if vis else str(local_rank)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(workload, with_gt=False):
    from paper_1805_03517_gb300 import synth

    pairs = [synth.make_pair(p.kind, p.seed, p.w, p.h) for p in workload.pairs]
    return pairs if with_gt else [pr[:2] for pr in pairs]


def flow_accuracy(flow, mask, gt):
    """End-point error of the forward field against the generated (integer) ground truth, as context: mean EPE
    over all pixels and over the matches kept by the consistency check, the share kept, and the share of
    outliers (EPE > 3 px and > 5 % of the ground-truth length, the KITTI 2015 rule)."""
    import numpy as np

    e = np.hypot(*(flow.astype(np.float64) - gt.astype(np.float64)).transpose(2, 0, 1))
    g = np.hypot(*gt.astype(np.float64).transpose(2, 0, 1))
    out = (e > 3.0) & (e > 0.05 * g)
    k = mask.astype(bool)
    return {"epe_all_px": float(e.mean()), "epe_kept_px": float(e[k].mean()) if k.any() else None,
            "kept_frac": float(k.mean()), "outliers_all": float(out.mean()),
            "outliers_kept": float(out[k].mean()) if k.any() else None}


def measure_batched(torch, ff, configs, stream, local_rank, steps, frames_call=True):
    """48 pairs of three sizes per step in merged launches (graph replay), inputs larger than L2; with frames_call,
    each step is one ff_match_frames call, else ff_features_batch + ff_match_batch."""
    wl = configs.workload("batch48_mixed")
    imgs = make_inputs(wl)
    dev = torch.device("cuda", local_rank)
    M = ff.Matcher(wl.pairs[0].params, local_rank, stream)
    with torch.cuda.stream(stream):
        d = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in imgs]
    stream.synchronize()
    pyrs = [(M.features(a), M.features(b)) for a, b in d]
    tuning = M.autotune(pyrs, reps=2)
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    outs = None

    frames = [x for pr in d for x in pr]

    def step():  # features of all 96 frames in one launch per kernel, then the merged matching launches
        nonlocal outs
        if frames_call:
            outs = M.match_frames(d, outs=outs, with_cost=False)
            return
        fp = M.features_batch(frames)
        pyrs = list(zip(fp[0::2], fp[1::2]))
        outs = M.match_batch(pyrs, outs=outs, with_cost=False)
        for p in fp:
            M.release(p)

    for _ in range(3):
        step()
    s0 = M.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("ff_batched")  # lets a profiler select exactly these timed steps
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = M.stats()["kernel_launches"] - s0["kernel_launches"]
    # propagation roofline of the batched step (its features, 5 GB, exceed L2): the level-0 launches, timed live in
    # a profiling context with the same launch configurations; DRAM bytes and L1 wavefronts per algorithmic byte
    # from the committed capture of an 8-pair KITTI batch (also beyond L2), scaled to this batch's launches
    P = ff.Matcher(wl.pairs[0].params, local_rank, stream)
    for lvl, cfg in enumerate(tuning):
        ff.ff_set_tuning(P.ctx, lvl, cfg)
    ff.ff_profile_enable(P.ctx, True)
    n_prof = 3
    for r in range(n_prof + 1):
        if r == 1:
            ff.ff_profile_read(P.ctx)
        fp = P.features_batch(frames)
        P.match_batch(list(zip(fp[0::2], fp[1::2])), with_cost=False)
        for p in fp:
            P.release(p)
    passes = ff.ff_profile_read_passes(P.ctx)
    P.close()
    M.close()
    peak, peak_kind = load_peaks()
    l0_ms, l0_n = passes.get(0, (0.0, 0))
    l0_launch_ms = l0_ms / l0_n
    l0_alg = sum(p.w * p.h for p in wl.pairs) * wl.pairs[0].params.iters * 2 * ALG_BYTES_PER_PIXEL_ITER / (l0_n / n_prof)
    alg_gbs = l0_alg / (l0_launch_ms / 1000.0) / 1e9
    roof = {"kernel": f"{prop_kernel(tuning[0])} (level-0 launches)", "avg_launch_ms": l0_launch_ms, "alg_bytes_per_launch": l0_alg,
            "alg_gbs": alg_gbs, "launches_per_step": l0_n / n_prof}
    rec = batch_traffic()
    if rec:
        dram = rec["dram_per_alg_byte"] * l0_alg
        dram_gbs = dram / (l0_launch_ms / 1000.0) / 1e9
        roof.update({"traffic": dram, "traffic_note": rec["note"],
                     "hbm": {"achieved": dram_gbs, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                             "frac": dram_gbs / peak}})
        if rec.get("wavefronts_per_alg_byte") and rec.get("wavefronts_peak_per_cycle"):
            clk = rec["sm_clock_hz"]
            wf = rec["wavefronts_per_alg_byte"] * l0_alg / (l0_launch_ms / 1000.0)
            roof.update({"bound": "l1", "unit": "wavefronts/s", "achieved": wf,
                         "peak": rec["wavefronts_peak_per_cycle"] * clk, "frac": wf / (rec["wavefronts_peak_per_cycle"] * clk),
                         "peak_kind": "ncu peak_sustained of l1tex__data_pipe_lsu_wavefronts x the captured SM clock"})
        else:
            roof.update({"bound": "hbm", "unit": "GB/s", "achieved": dram_gbs, "peak": peak, "frac": dram_gbs / peak})
    else:
        roof.update({"bound": "hbm", "unit": "GB/s", "achieved": alg_gbs, "peak": peak, "frac": alg_gbs / peak,
                     "traffic": None, "note": "algorithmic bytes; no DRAM capture for this kernel source"})
    return {"workload": wl.name, "pairs_per_step": len(wl.pairs), "px_per_step": wl.pixels,
            "value": wl.pixels / (ms / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "gpu_launches_per_step": launches / steps, "tiles_per_level": [list(c) for c in tuning],
            "l2": "not flushed: 5 GB of features per step exceed L2", "roofline": roof,
            "features": "ff_match_frames" if frames_call else "ff_features_batch + ff_match_batch"}


def measure_census(torch, ff, configs, stream, local_rank, steps, flush):
    """The Sintel-shaped 1024x436 pair matched with the Census cost (7x7 patterns, Hamming distance: the cost
    the paper takes for Sintel) and, for comparison, with the WHT-SAD cost; autotuned, L2 flushed per step."""
    import dataclasses

    wl = configs.workload("sintel_1024x436")
    spec = wl.pairs[0]
    imgs = make_inputs(wl)
    dev = torch.device("cuda", local_rank)
    with torch.cuda.stream(stream):
        d = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in imgs]
    stream.synchronize()
    peak, _ = load_peaks()
    out = {"workload": wl.name, "px_per_step": wl.pixels, "eps": spec.params.eps, "steps": steps,
           "l2": "flushed before every timed step"}
    for name, cost in (("census", 1), ("wht_sad", 0)):
        M = ff.Matcher(dataclasses.replace(spec.params, cost=cost), local_rank, stream)
        pyrs = [(M.features(a), M.features(b)) for a, b in d]
        tuning = M.autotune(pyrs, reps=2)
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)
        outs = None

        def step():
            nonlocal outs
            pyrs = [(M.features(a), M.features(b)) for a, b in d]
            outs = M.match_batch(pyrs, outs=outs, with_cost=False)
            for pa, pb in pyrs:
                M.release(pa)
                M.release(pb)

        for _ in range(3):
            step()
        ev = []
        for _ in range(steps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            ev.append((e0, e1))
        stream.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        # propagation roofline of this cost: algorithmic bytes per launch / device time per launch (profiling
        # context with the same launch configuration)
        P = ff.Matcher(dataclasses.replace(spec.params, cost=cost), local_rank, stream)
        for lvl, cfg in enumerate(tuning):
            ff.ff_set_tuning(P.ctx, lvl, cfg)
        ff.ff_profile_enable(P.ctx, True)
        n_prof = 10
        for r in range(n_prof + 2):
            if r == 2:
                ff.ff_profile_read(P.ctx)
            flush()
            pyrs = [(P.features(a), P.features(b)) for a, b in d]
            P.match_batch(pyrs, with_cost=False)
            for pa, pb in pyrs:
                P.release(pa)
                P.release(pb)
        prop_ms, prop_launches = ff.ff_profile_read(P.ctx)["propagate"]
        P.close()
        per_px_iter = ALG_BYTES_PER_PIXEL_ITER_CENSUS if cost else ALG_BYTES_PER_PIXEL_ITER
        pix_iters = ff.ff_work_counts(M.ctx, spec.w, spec.h)[0]
        bytes_per_launch = pix_iters * 2 * per_px_iter / (prop_launches / n_prof)
        achieved = bytes_per_launch / (prop_ms / prop_launches / 1000.0) / 1e9
        M.close()
        out[name] = {"value": wl.pixels / (ms / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": ms,
                     "tiles_per_level": [list(c) for c in tuning],
                     "k_propagate": {"alg_bytes_per_pixel_iter": per_px_iter, "achieved_gbs": achieved,
                                     "peak_gbs": peak, "frac": achieved / peak,
                                     "avg_launch_ms": prop_ms / prop_launches}}
    return out


def measure_filtered(torch, ff, configs, stream, local_rank, steps, flush, tuning):
    """The whole filter of Sec. 3.1 on the KITTI-shaped pair: forward field, two inverse fields (the second with
    its own random-search radius and hash stream), both consistency checks, then sparsification of what they
    left (3x3 blocks, s = 7 of Table 3); L2 flushed per step.  Also the sparsification kernel alone."""
    wl = configs.workload("kitti_1242x375")
    spec = wl.pairs[0]
    s_min = configs.TABLE3["kitti"]["min_matches"]
    imgs = make_inputs(wl)
    dev = torch.device("cuda", local_rank)
    with torch.cuda.stream(stream):
        d = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in imgs]
    stream.synchronize()
    M = ff.Matcher(spec.params, local_rank, stream)
    for lvl, cfg in enumerate(tuning):
        ff.ff_set_tuning(M.ctx, lvl, cfg)
    outs, sparse = None, None

    def step():
        nonlocal outs, sparse
        pyrs = [(M.features(a), M.features(b)) for a, b in d]
        outs = M.match_batch(pyrs, outs=outs, with_cost=False, second_check=True)
        with torch.cuda.stream(stream):
            sparse = [M.sparsify(o["flow_fwd"], o["flow_bwd"], spec.params.eps, s_min, keep=o["mask"]) for o in outs]
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)

    for _ in range(3):
        step()
    ev = []
    torch.cuda.nvtx.range_push("ff_filtered")  # lets a profiler select exactly these timed steps
    for _ in range(steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.nvtx.range_pop()
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    o = outs[0]
    # the sparsification kernel alone (inputs resident in L2: 10 algorithmic bytes per pixel -- forward flow,
    # the inverse flow at the target, the filter mask, the output): n_sp launches captured in a CUDA graph, so
    # the device time is not bounded by the host's launch rate
    n_sp, reps = 100, 20
    sp_out = torch.empty((spec.h, spec.w), dtype=torch.uint8, device=dev)
    sp_args = (o["flow_fwd"].data_ptr(), o["flow_bwd"].data_ptr(), o["mask"].data_ptr(), spec.w, spec.h,
               spec.params.eps, s_min, sp_out.data_ptr())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(n_sp):
            ff.ff_sparsify(M.ctx, *sp_args)
    with torch.cuda.stream(stream):
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
    stream.synchronize()
    sp_ms = e0.elapsed_time(e1) / (n_sp * reps)
    assert torch.equal(sp_out, sparse[0])
    del g
    peak, _ = load_peaks()
    sp_gbs = 10 * wl.pixels / (sp_ms / 1000.0) / 1e9
    kept_two = float(o["mask"].float().mean().item())
    kept_sparse = float(sparse[0].float().mean().item())
    M.close()
    return {"workload": wl.name, "px_per_step": wl.pixels, "eps": spec.params.eps, "min_matches": s_min,
            "rs_radius2": spec.params.rs_radius2, "steps": steps, "value": wl.pixels / (ms / 1000.0) / 1e6,
            "unit": UNIT, "ms_per_step": ms, "l2": "flushed before every timed step",
            "kept_after_two_checks": kept_two, "kept_after_sparsification": kept_sparse,
            "k_sparsify": {"ms": sp_ms, "alg_bytes_per_px": 10, "achieved_gbs": sp_gbs, "peak_gbs": peak,
                           "frac": sp_gbs / peak,
                           "note": "device time per launch from a CUDA graph of 100 launches; inputs L2-resident"}}


def measure_sub_scales(torch, ff, configs, stream, local_rank, steps, flush, tuning):
    """The KITTI-shaped pair matched with sub-scales and sub-sub-scales (every level below the coarsest first on
    the grids of every 4th and every 2nd pixel, then on every pixel; the reading of Sec. 3.1 the library takes),
    levels in the package table's configurations, grid passes autotuned; L2 flushed per step.  Mpx/s counts level-0 pixels, as for the
    plain schedule, so the two are comparable per frame pair."""
    import dataclasses

    wl = configs.workload("kitti_1242x375")
    spec = wl.pairs[0]
    imgs = make_inputs(wl)
    dev = torch.device("cuda", local_rank)
    with torch.cuda.stream(stream):
        d = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in imgs]
    stream.synchronize()
    out = {"workload": wl.name, "px_per_step": wl.pixels, "steps": steps, "l2": "flushed before every timed step"}
    for n_sub in (1, 2):
        M = ff.Matcher(dataclasses.replace(spec.params, sub_scales=n_sub), local_rank, stream)
        for lvl, cfg in enumerate(tuning):
            ff.ff_set_tuning(M.ctx, lvl, cfg)
        pyrs = [(M.features(a), M.features(b)) for a, b in d]
        M.autotune(pyrs, reps=2)  # configurations of the grid passes (the levels keep the table's)
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)
        outs = None

        def step():
            nonlocal outs
            pyrs = [(M.features(a), M.features(b)) for a, b in d]
            outs = M.match_batch(pyrs, outs=outs, with_cost=False)
            for pa, pb in pyrs:
                M.release(pa)
                M.release(pb)

        for _ in range(3):
            step()
        ev = []
        for _ in range(steps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            ev.append((e0, e1))
        stream.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        pix_iters = ff.ff_work_counts(M.ctx, spec.w, spec.h)[0]
        M.close()
        out[f"sub_scales_{n_sub}"] = {"value": wl.pixels / (ms / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": ms,
                                      "pixel_iters_per_direction": pix_iters}
    return out


def _make_pair_task(spec):
    from paper_1805_03517_gb300 import synth

    kind, seed, w, h = spec
    a, b, _ = synth.make_pair(kind, seed, w, h)
    return a, b


def measure_served(torch, ff, configs, stream, local_rank, n_req):
    """Served stream: Poisson arrivals (200 pairs/s) of n_req distinct frame pairs, each generated from its own seed
    with a size drawn uniformly from four sizes, continuous batching under a 60 GB device budget; latency from
    arrival to completion.  Also the same requests all arriving at once."""
    import multiprocessing as mp

    from paper_1805_03517_gb300 import serve

    dev = torch.device("cuda", local_rank)
    prm = configs.KITTI
    M = ff.Matcher(prm, local_rank, stream)
    specs = [configs.serve_pair(i) for i in range(n_req)]
    t_gen = time.perf_counter()
    frames = []
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        for a, b in pool.imap(_make_pair_task, [(p.kind, p.seed, p.w, p.h) for p in specs], chunksize=4):
            with torch.cuda.stream(stream):
                frames.append((torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)))
    stream.synchronize()
    gen_s = time.perf_counter() - t_gen
    for (w, h, _) in configs.SERVE_SIZES:  # per-size launch configurations, as a deployment would tune once:
        same = [f for f, p in zip(frames, specs) if (p.w, p.h) == (w, h)][:32]
        pyrs = [(M.features(a), M.features(b)) for a, b in same]
        M.autotune(pyrs[:1], reps=2)  # for one pair in flight (light load)
        M.autotune(pyrs, reps=2)      # for launches shared by many pairs (under load: 64 directions per size)
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)
    arrivals = serve.poisson_arrivals(n_req, 200.0, seed=5)
    serve.serve(M, frames[:512], [0.0] * 512)  # warm-up: pyramid and scratch pools at full occupancy, caches
    offered = serve.serve(M, frames, arrivals, mem_budget_bytes=60 << 30)
    saturated = serve.serve(M, frames, [0.0] * n_req, mem_budget_bytes=60 << 30)
    M.close()
    out = {"requests": n_req, "arrival_rate_per_s": 200.0, "sizes": [f"{w}x{h}" for w, h, _ in configs.SERVE_SIZES],
           "mem_budget_gb": 60,
           "inputs": f"{n_req} distinct synthetic pairs, pair i from seed 5000 + i (generated in {gen_s:.0f} s on "
                     "the host, resident on the device before the stream starts)",
           "offered_load": offered.as_dict(), "saturated": saturated.as_dict()}
    return out


def cpu_baseline(workload, imgs, cost_id=0):
    """The oracle as it stands, single-threaded, on one pair of the workload (a bounded sample)."""
    import oracle

    spec = workload.pairs[0]
    a, b = imgs[0]
    p = spec.params
    o = oracle.default()
    t = time.perf_counter()
    o.match_bidir(a, b, oracle.params(p.n_scales, p.iters, p.rs_radius, p.eps, p.seed, cost_id))
    dt = time.perf_counter() - t
    return {"value": spec.pixels / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one {spec.w}x{spec.h} pair of the workload, full bidirectional matching, "
                      f"{dt:.2f} s on 1 host thread"}


def _oracle_task(args):
    import oracle

    a, b, prm = args
    o = oracle.default()
    o.match_bidir(a, b, oracle.params(*prm))
    return a.shape[0] * a.shape[1]


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, as it stands, on the host cores; one pair per step, steps spread over a
    process pool (one single-threaded oracle per core)."""
    if rank != 0:
        return
    import multiprocessing as mp

    from paper_1805_03517_gb300 import configs

    workload = configs.workload(args.workload)
    imgs = make_inputs(workload)
    import oracle

    oracle.build()
    spec = workload.pairs[0]
    p = spec.params
    task = (imgs[0][0], imgs[0][1], (p.n_scales, p.iters, p.rs_radius, p.eps, p.seed, COSTS[args.cost]))
    cores = max(1, min(os.cpu_count() or 1, args.steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        if args.warmup:
            pool.map(_oracle_task, [task] * min(args.warmup, cores))
        t = time.perf_counter()
        px = sum(pool.map(_oracle_task, [task] * args.steps))
        dt = time.perf_counter() - t
    value = px / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1000 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload.name, "pairs_per_step": 1, "n_scales": p.n_scales, "iters": p.iters,
                       "cost": args.cost},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full {spec.w}x{spec.h} pairs over {cores} single-threaded "
                                       "oracle processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_1805_03517_gb300 import build as B
    from paper_1805_03517_gb300 import configs, ff

    B.build()
    workload = configs.workload(args.workload)
    imgs_gt = make_inputs(workload, with_gt=True)
    imgs = [pr[:2] for pr in imgs_gt]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    import dataclasses

    cost_id = COSTS[args.cost]
    prm = dataclasses.replace(workload.pairs[0].params, cost=cost_id)
    M = ff.Matcher(prm, local_rank, stream)
    with torch.cuda.stream(stream):
        dev_imgs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in imgs]
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream.synchronize()
    px_per_step = workload.pixels
    outs = None

    def features(m, imgs):
        if args.features == "batch":
            fp = m.features_batch([x for pr in imgs for x in pr])
            return list(zip(fp[0::2], fp[1::2]))
        return [(m.features(a), m.features(b)) for a, b in imgs]

    def match_step(m, imgs, outs):
        """One step's features and matching through the public API; returns the outputs."""
        if args.features == "frames":
            return m.match_frames(imgs, outs=outs, with_cost=False)
        pyrs = features(m, imgs)
        outs = m.match_batch(pyrs, outs=outs, with_cost=False)
        for pa, pb in pyrs:
            m.release(pa)
            m.release(pb)
        return outs

    ff.ff_set_option(M.ctx, ff.FF_OPT_OVERLAP, args.overlap)

    def step():
        nonlocal outs
        outs = match_step(M, dev_imgs, outs)

    def timed(n, body, pre=None):
        ms = []
        for _ in range(n):
            if pre:
                pre()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            body()
            e1.record(stream)
            ms.append((e0, e1))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    # per-level propagation configuration: given, from the package's table of autotuned configurations for this
    # workload, or chosen now by the library's autotuner (--autotune, or a workload without a table entry)
    table = {}
    with open(os.path.join(ROOT, "paper_1805_03517_gb300", "tuned.json")) as f:
        table = json.load(f)
    tuning_source = "autotuned in this run"
    if args.tuning or (workload.name in table and not args.autotune and cost_id == 0):
        tuning = [tuple(c) for c in (json.loads(args.tuning) if args.tuning else table[workload.name])]
        tuning_source = "given" if args.tuning else "package table of ff_autotune results on GB300"
        for lvl, cfg in enumerate(tuning):
            ff.ff_set_tuning(M.ctx, lvl, cfg)
    else:
        pyrs = [(M.features(a), M.features(b)) for a, b in dev_imgs]
        tuning = M.autotune(pyrs, reps=3)
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)
    stream.synchronize()

    # untimed steps until the GPU has been busy for --settle-s seconds (its clocks ramp up under sustained load
    # on a freshly started process), then the W warm-up steps
    t_settle = time.perf_counter()
    while time.perf_counter() - t_settle < args.settle_s:
        for _ in range(50):
            flush_l2()
            step()
        stream.synchronize()
    for _ in range(args.warmup):
        flush_l2()
        step()
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    s0 = M.stats()
    sampler = ClockSampler(local_rank)
    sampler.start()
    torch.cuda.nvtx.range_push("ff_timed")  # lets a profiler select exactly the timed steps
    times = timed(args.steps, step, pre=flush_l2)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    s1 = M.stats()
    if dist:
        dist.barrier()
    ms, value = aggregate_ranks(torch, dist, dev, sum(times) / len(times), px_per_step, world)
    launches = int(s1["kernel_launches"] - s0["kernel_launches"])

    # end to end through the public API, copies inside the timing: every step's frames go from one pinned host
    # buffer to the device in one copy, and its result (forward and inverse flows and mask of every pair) comes
    # back in one copy (each frame and output starts on a 256-byte boundary of its buffer)
    def packed(sizes):
        offs, total = [], 0
        for n in sizes:
            offs.append(total)
            total += (n + 255) // 256 * 256
        return offs, total

    in_offs, in_total = packed([x.nbytes for pr in imgs for x in pr])
    h_in = torch.empty(in_total, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(in_total, dtype=torch.uint8, device=dev)
    e2e_imgs = []
    for i, (a, b) in enumerate(imgs):
        views = []
        for x, off in zip((a, b), in_offs[2 * i:2 * i + 2]):
            h_in[off:off + x.nbytes].copy_(torch.from_numpy(x).reshape(-1))
            views.append(d_in[off:off + x.nbytes].view(x.shape))
        e2e_imgs.append(tuple(views))
    out_shapes = []
    for p in workload.pairs:
        out_shapes += [("flow_fwd", (p.h, p.w, 2), torch.int16), ("flow_bwd", (p.h, p.w, 2), torch.int16),
                       ("mask", (p.h, p.w), torch.uint8)]
    out_bytes = [math.prod(sh) * torch.tensor([], dtype=dt).element_size() for _, sh, dt in out_shapes]
    out_offs, out_total = packed(out_bytes)
    d_out = torch.empty(out_total, dtype=torch.uint8, device=dev)
    h_out = torch.empty(out_total, dtype=torch.uint8).pin_memory()
    e2e_outs = [{} for _ in workload.pairs]
    for j, ((k, sh, dt), off, nb) in enumerate(zip(out_shapes, out_offs, out_bytes)):
        e2e_outs[j // 3][k] = d_out[off:off + nb].view(dt).view(sh)

    def e2e_step():
        with torch.cuda.stream(stream):
            d_in.copy_(h_in, non_blocking=True)
        match_step(M, e2e_imgs, e2e_outs)
        with torch.cuda.stream(stream):
            h_out.copy_(d_out, non_blocking=True)

    for _ in range(3):
        e2e_step()
    e2e_times = timed(max(10, args.steps // 4), e2e_step, pre=flush_l2)
    e2e_ms = sum(e2e_times) / len(e2e_times)
    h2d, d2h = in_total, out_total
    for o, eo in zip(outs, e2e_outs):  # the end-to-end result equals the device-timed one
        for k in ("flow_fwd", "flow_bwd", "mask"):
            assert torch.equal(o[k], eo[k]), k

    # per-phase device time (profiling context: same kernels and launch shapes, phases bracketed by events)
    P = ff.Matcher(prm, local_rank, stream)
    for lvl, cfg in enumerate(tuning):
        ff.ff_set_tuning(P.ctx, lvl, cfg)
    ff.ff_profile_enable(P.ctx, True)
    prof_outs = None

    def prof_step():
        nonlocal prof_outs
        prof_outs = match_step(P, dev_imgs, prof_outs)

    for _ in range(3):
        prof_step()
    ff.ff_profile_read(P.ctx)
    n_prof = max(5, min(50, args.steps))
    for _ in range(n_prof):
        flush_l2()
        prof_step()
    phases = ff.ff_profile_read(P.ctx)
    for _ in range(n_prof):
        flush_l2()
        prof_step()
    passes = ff.ff_profile_read_passes(P.ctx)
    P.close()
    pix_iters = sum(ff.ff_work_counts(M.ctx, p.w, p.h)[0] for p in workload.pairs)
    prop_ms, prop_launches = phases["propagate"]
    alg_bytes_per_step = pix_iters * 2 * (ALG_BYTES_PER_PIXEL_ITER_CENSUS if cost_id else ALG_BYTES_PER_PIXEL_ITER)
    launches_per_step = prop_launches / n_prof
    avg_launch_ms = prop_ms / prop_launches
    bytes_per_launch = alg_bytes_per_step / launches_per_step
    achieved = bytes_per_launch / (avg_launch_ms / 1000.0) / 1e9
    peak, peak_kind = load_peaks()
    # level 0, the dominant launches: algorithmic bytes and live device time per launch
    l0_ms, l0_launches = passes.get(0, (0.0, 0))
    l0_px_iters = sum(p.w * p.h for p in workload.pairs) * prm.iters * 2
    l0_launch_ms = l0_ms / l0_launches if l0_launches else None
    l0_alg = l0_px_iters * (ALG_BYTES_PER_PIXEL_ITER_CENSUS if cost_id else ALG_BYTES_PER_PIXEL_ITER) / (
        l0_launches / n_prof) if l0_launches else None
    hbm_roof = {"bound": "hbm", "kernel": "propagation, all levels: " + ", ".join(
                    sorted({prop_kernel(c) for c in tuning})), "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": achieved / peak,
                "traffic": propagate_traffic(tuning) if cost_id == 0 else None,
                "alg_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_launch_ms,
                "launches_per_step": launches_per_step}
    rec = propagate_l1_record(tuning) if cost_id == 0 and workload.name == "kitti_1242x375" else None
    if rec and l0_launch_ms and clocks.get("sm_mhz"):
        # what binds (ncu): the L1 LSU data-pipe wavefront rate of the scattered 32-byte descriptor gathers; peak =
        # ncu's sustained wavefronts per cycle (whole GPU) x the SM clock sampled during the timed steps
        wf_peak = rec["wavefronts_peak_per_cycle"] * clocks["sm_mhz"] * 1e6
        wf_achieved = rec["wavefronts_per_launch"] / (l0_launch_ms / 1000.0)
        share = (l0_ms / n_prof) / ms
        roofline = {"bound": "l1", "kernel": f"{prop_kernel(tuning[0])} (level-0 launches, {100 * share:.0f} % of a step)",
                    "unit": "wavefronts/s", "achieved": wf_achieved, "peak": wf_peak,
                    "peak_kind": "ncu peak_sustained of l1tex__data_pipe_lsu_wavefronts x sampled SM clock",
                    "frac": wf_achieved / wf_peak, "traffic": rec["dram_bytes_per_launch"],
                    "traffic_unit": "DRAM bytes per level-0 launch (ncu)", "avg_launch_ms": l0_launch_ms,
                    "alg_bytes_per_launch": l0_alg,
                    "ncu": {k: rec[k] for k in ("l1_wavefront_pct", "l1_hit_pct", "l2_hit_pct", "capture")},
                    "hbm": {"achieved": l0_alg / (l0_launch_ms / 1000.0) / 1e9, "peak": peak, "peak_kind": peak_kind,
                            "unit": "GB/s", "frac": l0_alg / (l0_launch_ms / 1000.0) / 1e9 / peak,
                            "dram_gbs": rec["dram_bytes_per_launch"] / (l0_launch_ms / 1000.0) / 1e9,
                            "dram_frac": rec["dram_bytes_per_launch"] / (l0_launch_ms / 1000.0) / 1e9 / peak},
                    "all_levels": hbm_roof}
    else:
        roofline = hbm_roof

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int16", "data": "synthetic",
            "config": {"workload": workload.name, "pairs_per_step": len(workload.pairs),
                       "px_per_step": px_per_step, "n_scales": prm.n_scales, "iters": prm.iters,
                       "rs_radius": prm.rs_radius, "eps": prm.eps, "cost": args.cost,
                       "parallelism": f"replicas x{world}",
                       "tiles_per_level": {str(l): list(c) for l, c in enumerate(tuning)},
                       "tiles_from": tuning_source,
                       "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MiB write, outside the events)",
                       "features": {"batch": "ff_features_batch (one launch per kernel for all frames)",
                                    "frame": "ff_features per frame",
                                    "frames": "ff_match_frames (features and matching in one call; levels 0-1 "
                                              f"descriptors on a branch of the matching graph, FF_OPT_OVERLAP {args.overlap})"
                                    }[args.features],
                       "settle_s": args.settle_s},
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": {"value": px_per_step * world / (e2e_ms / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "propagate_ms_per_pass": {str(k): v[0] / n_prof for k, v in sorted(passes.items())},
            "phases_ms_per_step": {k: v[0] / n_prof for k, v in phases.items()},
            "accuracy_context": flow_accuracy(outs[0]["flow_fwd"].cpu().numpy(), outs[0]["mask"].cpu().numpy(),
                                              imgs_gt[0][2]),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(workload, imgs, cost_id)
    if not args.no_filtered and workload.name == "kitti_1242x375" and cost_id == 0:
        try:  # an auxiliary measurement: report its failure in the line instead of losing the line
            filtered = measure_filtered(torch, ff, configs, stream, local_rank, max(10, min(100, args.steps // 3)),
                                        flush_l2, tuning)
        except Exception as e:  # noqa: BLE001
            filtered = {"error": repr(e)}
        if rank == 0:
            line["filtered"] = filtered
    if not args.no_sub_scales and workload.name == "kitti_1242x375" and cost_id == 0:
        try:  # an auxiliary measurement: report its failure in the line instead of losing the line
            sub = measure_sub_scales(torch, ff, configs, stream, local_rank, max(10, min(100, args.steps // 3)),
                                     flush_l2, tuning)
        except Exception as e:  # noqa: BLE001
            sub = {"error": repr(e)}
        if rank == 0:
            line["sub_scales"] = sub
    if not args.no_census:
        census = measure_census(torch, ff, configs, stream, local_rank, max(10, min(100, args.steps // 3)), flush_l2)
        if rank == 0:
            line["census_cost"] = census
    if not args.no_batched:
        batched = measure_batched(torch, ff, configs, stream, local_rank, steps=max(5, min(30, args.steps // 10)),
                                  frames_call=args.features == "frames")
        if rank == 0:
            line["batched"] = batched
    if not args.no_served:
        served = measure_served(torch, ff, configs, stream, local_rank, args.serve_requests)
        if rank == 0:
            line["served"] = served
    if rank == 0:
        print(json.dumps(line), flush=True)
    M.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
