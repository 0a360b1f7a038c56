#!/usr/bin/env python
"""Throughput of the whole HR-EBSD hot path on GB300, in pattern pairs per second.

One step = one pass of every stage over one batch of synthetic pairs:
preprocess (references + tests), multi-resolution demons registration,
rotation fit, remap, second-pass ROI XCF and deformation-gradient solve, all
through the C ABI of libhrebsd.  Workload (default): the batched scan of
100 x 100 = 10,000 test patterns at 256 x 256 FP32 against 4 grain
references, demons with 4 levels and a convergence-driven stop (<= 100
iterations per level), 25 ROIs of 64 x 64.  Inputs come from the seeded
Kikuchi generator and are resident in HBM before timing (2.6 GB, larger than
L2, so no flush is needed between steps).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank processes its own 10,000 pairs (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl reference
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ALGO_BYTES_PER_PIXEL_ITER = 24   # test 4 B + moving 4 B + field 8 B read, field 8 B written
FALLBACK_HBM_GBS = 6800.0
METRIC = "pattern pairs/s (demons+XCF) on 1 GB300"


def workload(n_pairs):
    from synth import kikuchi as K
    spec = K.config2(n_pairs)
    return dict(spec=spec, H=256, W=256, levels=4, caps=(100, 100, 100, 100), stop_window=5, stop_tol=1e-4,
                S=64, roi=K.roi_grid(256, 256, 64, False))


def workload_config(wl, B):
    return {"workload": f"batched scan: {B} test patterns 256x256 FP32 vs 4 grain references; demons 4 levels, "
                        f"<=100 it/level, stop w=5 tol=1e-4, alpha=1, sigma=1; 25 ROIs 64x64; FP64 fits",
            "pairs_per_gpu": B, "H": 256, "W": 256, "refs": 4, "levels": 4, "max_iters_per_level": 100,
            "rois": 25, "roi_size": 64, "misorientation_deg": [0, 6], "counts": 500,
            "l2": "inputs (2.6 GB) larger than L2; no flush"}


# ------------------------------------------------------------------ oracle on host cores
def _oracle_pair(args):
    p, n_pairs = args
    import numpy as np
    import oracle
    from synth import kikuchi as K
    wl = workload(n_pairs)
    spec = wl["spec"]
    r = K.ref_index(spec, p)
    ref = K.render_ref(spec, r).astype(np.float64)
    test = K.render_test(spec, p).astype(np.float64)
    t0 = time.perf_counter()
    oracle.pipeline(ref, test, wl["roi"], wl["S"], spec.geom, wl["levels"], list(wl["caps"]), 1.0, 1.0,
                    wl["stop_window"], wl["stop_tol"])
    return time.perf_counter() - t0


def oracle_throughput(n_sample, n_pairs, cores, pool=None):
    """Pairs/s of the oracle over `n_sample` pairs, one pair per process."""
    import oracle
    oracle.build()
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    try:
        t0 = time.perf_counter()
        per_pair = pool.map(_oracle_pair, [(p, n_pairs) for p in range(n_sample)], chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    return n_sample / wall, sum(per_pair), wall


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d and isinstance(d[k], (int, float)):
                return float(d[k]), "measured"
        for v in d.values():
            if isinstance(v, dict) and "hbm_gbs" in v:
                return float(v["hbm_gbs"]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def xcf_roofline(ms, B, wl, fp32_peak_tflops, hbm_peak):
    """ROI cross-correlation against the FP32 FMA peak (probe) and HBM.  Algorithmic work
    per ROI of S x S: one packed complex forward FFT and one inverse (5 S^2 log2 S^2 each)
    plus ~20 S^2 for the cross power and unpacking; bytes: both ROIs read, 2 S^2 x 4 B."""
    import math
    S, N = wl["S"], len(wl["roi"])
    flops = B * N * (2 * 5 * S * S * math.log2(S * S) + 20 * S * S)
    nbytes = B * N * 2 * S * S * 4
    t = ms / 1e3
    return {"kernel": "xcf64_kernel", "ms_per_step": ms,
            "tflops": flops / t / 1e12, "fp32_peak_tflops_probe": fp32_peak_tflops,
            "frac_fp32": flops / t / 1e12 / fp32_peak_tflops,
            "gbs": nbytes / t / 1e9, "frac_hbm": nbytes / t / 1e9 / hbm_peak,
            "algorithmic": f"{flops / B / 1e6:.2f} MFLOP and {nbytes / B / 1e3:.0f} KB per pair"}


def code_digest(*paths):
    """SHA-256 of C/CUDA sources (in the order given) with their // comments, trailing blanks and empty
    lines removed: a change of the code (not of its comments) changes it.  The demons sources hold no
    '//' inside string literals."""
    lines = []
    for path in paths:
        for line in open(path, encoding="utf-8").read().splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def demons_sources():
    csrc = os.path.join(ROOT, "paper_1907_05993_gb300", "csrc")
    return os.path.join(csrc, "demons.cu"), os.path.join(csrc, "demons_strip.cuh")


def traffic_per_launch(px_per_launch):
    """DRAM bytes per demons-iteration launch from the committed ncu summary, if the kernel's code is
    still the one that was captured."""
    path = os.path.join(ROOT, "profiles", "demons_iter_traffic.json")
    try:
        d = json.load(open(path))
        if d.get("demons_code_sha256") != code_digest(*demons_sources()):
            return None
        return d["dram_bytes_per_pixel_iter"] * px_per_launch
    except Exception:
        return None


# ------------------------------------------------------------------ main arms
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = workload(args.pairs)
    cores = os.cpu_count() or 1
    sample = max(cores, args.ref_sample)
    pool = mp.get_context("spawn").Pool(cores)
    try:
        for _ in range(args.warmup):
            oracle_throughput(min(sample, cores), args.pairs, cores, pool)
        vals, cpu_s = [], 0.0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, cs, wall = oracle_throughput(sample, args.pairs, cores, pool)
            vals.append(wall)
            cpu_s += cs
        total = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = args.steps * sample / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.pairs),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} pairs of the workload per step (pairs 0..{sample - 1}), "
                                       f"one pair per process, FP64 C oracle"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


E2E_CHUNKS, E2E_GROWTH = 2, 4.0   # slices of the end-to-end (host-buffer) path: 1 : 4


def run_ours(args, rank, world, local_rank):
    cpu = None
    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not (args.no_cpu_baseline and args.no_learned):
        # before any CUDA call: the oracle pool is spawned, never forked from a CUDA process
        import oracle
        oracle.build()
        pool = mp.get_context("spawn").Pool(cores)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = max(cores, args.cpu_sample)
        v, cpu_s, wall = oracle_throughput(n, args.pairs, cores, pool)
        cpu = {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} pairs of the workload (pairs 0..{n - 1}), one pair per process over {cores} host "
                         f"cores, {cpu_s:.1f} s of CPU work"}
    import numpy as np
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as synth_gpu

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = workload(args.pairs)
    spec = wl["spec"]
    B = args.pairs
    # this rank's shard of a world * B point scan (independent pairs)
    from synth import kikuchi as K
    from paper_1907_05993_gb300.shard import max_over_ranks, shard_range
    spec = K.ScanSpec(**{**spec.__dict__, "n_pairs": B * world})
    pairs = shard_range(B * world, rank, world)
    refs, tests, ridx, _ = synth_gpu.make_scan_gpu(spec, pairs)
    torch.cuda.synchronize()
    cfg = PipelineConfig(wl["H"], wl["W"], wl["roi"], wl["S"], wl["levels"], wl["caps"], 1.0, 1.0,
                         wl["stop_tol"], wl["stop_window"], autotune=args.tile_variants is None)
    pipe = Pipeline(cfg, device=local_rank)
    if args.tile_variants is not None:   # fixed tile shapes per level (finest first), no autotuning
        for l, v in enumerate(args.tile_variants[:wl["levels"]]):
            P.hrebsd_set_tile_variant(pipe.ctx, wl["H"] >> l, wl["W"] >> l, v)
    stream = torch.cuda.current_stream()
    out = {}
    for _ in range(args.warmup):
        pipe.run(refs, tests, ridx, out=out)
    torch.cuda.synchronize()

    # ---- device-resident timing (tracing off: every pyramid level replays its cached CUDA graph)
    l0 = P.hrebsd_launch_count(pipe.ctx)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pipe.run(refs, tests, ridx, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = P.hrebsd_launch_count(pipe.ctx) - l0
    # ---- traced pass of the same steps: per-kernel CUDA events on the launch stream (the graphs carry
    # no per-kernel events, so the breakdown and the roofline of the demons iteration come from here)
    trace_steps = max(1, min(args.steps, 3))
    P.hrebsd_profile_enable(pipe.ctx, True)
    tr0, tr1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tr0.record(stream)
    for _ in range(trace_steps):
        pipe.run(refs, tests, ridx, out=out)
    tr1.record(stream)
    torch.cuda.synchronize()
    prof = P.hrebsd_profile_read(pipe.ctx)
    P.hrebsd_profile_enable(pipe.ctx, False)
    traced_ms_per_step = tr0.elapsed_time(tr1) / trace_steps
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, device="cuda")
    value = world * B * args.steps / t
    tune_ms = pipe._tuned.get((B, wl["H"], wl["W"]))

    def shape_name(v):
        if v == 5:
            return "row sweep/w threads"
        if v == 6:
            return "row sweep, one launch per level/w threads"
        if v == 7:
            return "level in shared memory/512t"
        return "x".join(map(str, P.TILE_SHAPES[v])) + f"/{P.TILE_THREADS[v]}t"
    tile_choice = [
        {"level": l, "shape": shape_name(P.hrebsd_get_tile_variant(pipe.ctx, wl["H"] >> l, wl["W"] >> l)),
         **({"pinned": True} if tune_ms is None else
            {"ms_per_iteration_by_shape": {shape_name(v): round(float(tune_ms[l, v]), 4)
                                           for v in range(P.TILE_VARIANTS) if np.isfinite(tune_ms[l, v])}})}
        for l in range(wl["levels"])]
    iters = out["iters"].cpu().numpy()
    status = out["status"].cpu().numpy()

    # ---- end to end through the ABI with host buffers (pinned), copies inside the timed region
    h_tests = tests.cpu().pin_memory()
    h_refs = refs.cpu().pin_memory()
    h_ridx = ridx.cpu().pin_memory()
    h_F = torch.empty((B, 9), dtype=torch.float64).pin_memory()
    h_R = torch.empty((B, 9), dtype=torch.float64).pin_memory()
    h_st = torch.empty((B,), dtype=torch.int32).pin_memory()
    e_steps = max(1, min(args.steps, 3))
    # Pipeline.run_host: the batch in E2E_CHUNKS slices of growing size, the host -> device copy of slice k + 1 on a
    # side stream while slice k is processed, results copied back into pinned host tensors.  One
    # untimed pass first (new slice buffers: autotune and per-level graph capture happen there).
    host_out = {"F": h_F, "R_finite": h_R, "status": h_st}
    pipe.run_host(h_refs, h_tests, h_ridx, chunks=E2E_CHUNKS, out=host_out, growth=E2E_GROWTH)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        pipe.run_host(h_refs, h_tests, h_ridx, chunks=E2E_CHUNKS, out=host_out, growth=E2E_GROWTH)
    e1.record(stream)
    torch.cuda.synchronize()
    te = max_over_ranks(e0.elapsed_time(e1) / 1e3, device="cuda")
    if dist:
        dist.barrier()
    h2d = tests.numel() * 4 + refs.numel() * 4 + ridx.numel() * 4
    d2h = B * 9 * 8 * 2 + B * 4

    # FP32 FMA throughput of this GPU (probe kernel), the ALU peak of the XCF roofline
    P.hrebsd_probe_fp32_fma(pipe.ctx, 256)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    probe_flops = sum(P.hrebsd_probe_fp32_fma(pipe.ctx, 4096) for _ in range(3))
    p1.record(stream)
    torch.cuda.synchronize()
    fp32_peak = probe_flops / (p0.elapsed_time(p1) / 1e3) / 1e12
    pipe.close()

    # learned initialiser vs plain on the learned-vs-plain scan (rank 0 of a 1-GPU run; network trained here
    # on a reduced set so that the run stays within minutes; --workload learned uses the full recipe)
    lvp = None
    if pool is not None and not args.no_learned:
        del refs, tests, out
        torch.cuda.empty_cache()
        lvp = learned_comparison(args, local_rank, pool, args.lvp_train_pairs, args.lvp_epochs, args.pairs,
                                 args.oracle_pairs, max(3, args.warmup), max(1, min(args.steps, 3)))
        lvp["training"]["note"] += (f"; reduced set for the default benchmark ({args.lvp_train_pairs} pairs, "
                                    f"{args.lvp_epochs} epochs; the full recipe is --workload learned)")
    if pool is not None:
        pool.close()
        pool.join()
    # latency of one pair through the whole chain (the single-pair workload), rank 0 of a 1-GPU run
    single = None
    if world == 1 and not args.no_single:
        sp = single_pair_latency(local_rank)
        single = {"workload": "1 pair 128x128, 2 deg, 3 levels x 50 iterations, 21 ROIs 32x32",
                  "ms_per_pair_graphs": sp[1][0], "ms_per_pair_direct": sp[0][0],
                  "kernel_launches_per_pair": sp[1][1]}

    if rank == 0:
        it = prof["demons_iter"]
        px = prof["pixel_iters"]
        peak, peak_kind = measured_peak_hbm()
        achieved = ALGO_BYTES_PER_PIXEL_ITER * px / (it["ms"] / 1e3) / 1e9 if it["ms"] > 0 else None
        px_per_launch = px / max(1, it["launches"])
        traffic = traffic_per_launch(px_per_launch)
        total_ms = sum(v["ms"] for k, v in prof.items() if k != "pixel_iters")
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded kinematic Kikuchi generator)",
            "config": workload_config(wl, B),
            "e2e": {"value": world * B * e_steps / te, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "path": f"Pipeline.run_host: pinned host inputs, {E2E_CHUNKS} slices of sizes 1:{E2E_GROWTH:g}, copy "
                            f"of slice k+1 overlapping slice k, F/R/status back to pinned host"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": "demons iteration (every launch of every level; shapes in "
                                                   "demons_tile_shape_per_level)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "algorithmic_bytes": f"{ALGO_BYTES_PER_PIXEL_ITER} B per pixel-iteration x "
                                              f"{px_per_launch:.0f} pixel-iterations per launch (average)",
                         "avg_launch_ms": it["ms"] / max(1, it["launches"]),
                         "share_of_step": it["ms"] / total_ms if total_ms else None},
            "xcf_roofline": xcf_roofline(prof["xcf"]["ms"] / trace_steps, B, wl, fp32_peak, peak),
            "kernel_ms_per_step": {k: v["ms"] / trace_steps for k, v in prof.items() if k != "pixel_iters"},
            "traced_pass": {"steps": trace_steps, "ms_per_step": traced_ms_per_step,
                            "note": "per-kernel CUDA events around every launch (direct launches, no graphs); "
                                    "the roofline and kernel_ms_per_step come from it"},
            "demons_tile_shape_per_level": tile_choice,
            "demons_iters_mean_per_level": [float(x) for x in iters.mean(axis=0)],
            "pairs_capped": int(np.sum(status & 1)),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if single is not None:
            line["single_pair_latency"] = single
        if lvp is not None:
            line["learned_vs_plain"] = lvp
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ learned initialiser vs plain
LEARNED_SCAN_PAIRS = 160_000   # the learned-init vs plain scan: 400 x 400 points, 8 grains, mis U(0, 12) deg


def _render5(p):
    from synth import kikuchi as K
    spec = K.config5(LEARNED_SCAN_PAIRS)
    return K.render_test(spec, p)


def _oracle5(args):
    """The oracle's chain on one config-5 pair: its own stop rule (replay None) or replaying the given
    per-level counts.  Returns (R_finite, F, iters)."""
    p, replay = args
    import numpy as np
    import oracle
    from synth import kikuchi as K
    spec = K.config5(LEARNED_SCAN_PAIRS)
    ref = K.render_ref(spec, K.ref_index(spec, p)).astype(np.float64)
    test = K.render_test(spec, p).astype(np.float64)
    res = oracle.pipeline(ref, test, K.roi_grid(256, 256, 64, False), 64, spec.geom, 4, [100] * 4, 1.0, 1.0, 5, 1e-4,
                          replay=replay)
    return res["R_finite"], res["F"], np.asarray(res["iters"])


def learned_comparison(args, local_rank, pool, train_pairs, epochs, n_points, oracle_pairs, warmup, steps):
    """Config-5 scan, first n_points points: plain registration (caps 100 x 4) vs registration started
    from the learned initialiser's field (args.learned_caps) vs a plain control with the learned run's
    fine-level caps; the network is trained first on train_pairs config-4 pairs for `epochs` epochs.
    A seeded subset of oracle_pairs points is rendered by the numpy generator on both sides and run by
    the oracle twice: with its own stop rule (the method's answer) and replaying the plain run's
    per-level counts (parity of the plain arm)."""
    import numpy as np
    import oracle as O
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300 import learned as LN
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as SG
    from synth import kikuchi as K
    rng = np.random.default_rng(505)
    sub = sorted(rng.choice(n_points, oracle_pairs, replace=False).tolist())
    t0 = time.perf_counter()
    own = pool.map(_oracle5, [(p, None) for p in sub], chunksize=2)
    renders = pool.map(_render5, sub, chunksize=8)
    t_oracle = time.perf_counter() - t0
    torch.cuda.set_device(local_rank)
    spec5 = K.config5(LEARNED_SCAN_PAIRS)
    refs, tests, ridx, F_true = SG.make_scan_gpu(spec5, range(n_points))
    refs = torch.from_numpy(np.stack([K.render_ref(spec5, r) for r in range(spec5.n_refs)])).cuda()
    for p, img in zip(sub, renders):
        tests[p] = torch.from_numpy(img).cuda()
    roi = K.roi_grid(256, 256, 64, False)
    pipe = Pipeline(PipelineConfig(256, 256, roi, 64, 4, (100, 100, 100, 100), 1.0, 1.0, 1e-4, 5),
                    device=local_rank)
    t0 = time.perf_counter()
    x, y = LN.build_training_set(pipe.ctx, K.config4(train_pairs))
    torch.cuda.synchronize()
    t_set = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = LN.train(pipe.ctx, x, y, epochs=epochs, batch=256, lr=args.lr, seed=0, lr_final=args.lr_final)
    del x, y
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    caps_l = tuple(args.learned_caps)
    ctrl_caps = (caps_l[0], caps_l[1], 100, 100)
    stream = torch.cuda.current_stream()

    def timed(learned, plain_caps=None):
        out = {}
        kw = {"learned_caps": caps_l, "learned_start_res": args.learned_start} if learned else {}
        saved = pipe.params
        if plain_caps is not None:
            pipe.params = P.demons_params(4, plain_caps, 1.0, 1.0, 1.0, 1e-4, 5)
        for _ in range(warmup):
            pipe.run(refs, tests, ridx, out=out, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            pipe.run(refs, tests, ridx, out=out, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        pipe.params = saved
        return (n_points * steps / t, out["R_finite"].cpu().numpy().reshape(-1, 3, 3),
                out["iters"].cpu().numpy())

    v_plain, R_plain, it_plain = timed(False)
    v_learn, R_learn, it_learn = timed(True)
    v_ctrl, R_ctrl, it_ctrl = timed(False, ctrl_caps)
    pipe.close()
    t0 = time.perf_counter()
    rep = pool.map(_oracle5, [(p, it_plain[p].astype(np.int32)) for p in sub], chunksize=2)
    t_oracle += time.perf_counter() - t0

    def rot_deg(Ra, Rb):
        M = np.asarray(Ra).T @ np.asarray(Rb)
        v = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2
        return float(np.degrees(np.arcsin(min(1.0, float(np.linalg.norm(v))))))

    def stats(e):
        e = np.asarray(e)
        return {"median": float(np.median(e)), "p95": float(np.percentile(e, 95)), "max": float(e.max()),
                "frac_le_1e-4_deg": float(np.mean(e <= 1e-4))}
    R_own = [o[0] for o in own]
    R_rep = [r[0] for r in rep]
    R_true = [O.polar(f) for f in F_true]
    dev = {name: [rot_deg(R[p], Ro) for p, Ro in zip(sub, R_own)]
           for name, R in (("plain", R_plain), ("learned", R_learn), ("control", R_ctrl))}
    dev_rep_plain = [rot_deg(R_plain[p], Ro) for p, Ro in zip(sub, R_rep)]
    truth = {name: [rot_deg(R[p], R_true[p]) for p in range(n_points)]
             for name, R in (("plain", R_plain), ("learned", R_learn), ("control", R_ctrl))}
    stop_d = np.abs(np.stack([it_plain[p] for p in sub]) - np.stack([o[2] for o in own]))
    f_plain = stats(dev["plain"])["frac_le_1e-4_deg"]
    f_learn = stats(dev["learned"])["frac_le_1e-4_deg"]
    holds = bool(v_learn > v_plain and f_learn >= f_plain)
    return {
        "workload": f"config-5 scan (400x400 points, 256x256, 8 grains, mis U(0,12) deg), first {n_points} points",
        "plain": {"caps": [100] * 4, "pairs_per_s": v_plain,
                  "iters_mean_per_level": [float(a) for a in it_plain.mean(axis=0)]},
        "learned": {"caps": list(caps_l), "start": f"{args.learned_start}x{args.learned_start} from the network's "
                                                 f"64x64 field", "pairs_per_s": v_learn,
                    "iters_mean_per_level": [float(a) for a in it_learn.mean(axis=0)]},
        "control_plain_same_fine_caps": {"caps": list(ctrl_caps), "pairs_per_s": v_ctrl,
                                         "iters_mean_per_level": [float(a) for a in it_ctrl.mean(axis=0)]},
        "speedup_learned_over_plain": v_learn / v_plain, "speedup_learned_over_control": v_learn / v_ctrl,
        "oracle_subset": {"pairs": len(sub), "seconds": t_oracle,
                          "inputs": "numpy-rendered on both sides (seeded subset, rng 505)"},
        "rot_dev_vs_oracle_own_stop_deg": {k: stats(v) for k, v in dev.items()},
        "rot_dev_plain_vs_oracle_replayed_deg": stats(dev_rep_plain),
        "stop_rule_plain_vs_oracle": {"exact": float(np.mean(stop_d == 0)), "within_1": float(np.mean(stop_d <= 1))},
        "rot_err_vs_ground_truth_deg": {k: stats(v) for k, v in truth.items()},
        "criterion": "learned-init beats plain in pairs/s at the same <= 1e-4 deg rotation error against the oracle "
                     "(fraction of the subset within 1e-4 deg of the oracle's own-stop answer at least the plain arm's)",
        "criterion_holds": holds,
        "training": {"pairs": train_pairs, "epochs": epochs, "seconds": t_train, "set_seconds": t_set,
                     "loss_first_last": [hist[0], hist[-1]],
                     "note": "trained in the benchmark run (config-4 recipe: 128x128, mis U(0,12) deg, target = final "
                             "field of the full registration at 64x64; Adam, batch 256, cosine step size)"},
    }


def run_learned(args, rank, world, local_rank):
    """The learned-init vs plain comparison with the full training recipe (config 4: 200,000 pairs)."""
    cores = os.cpu_count() or 1
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = learned_comparison(args, local_rank, pool, args.train_pairs, args.epochs, args.pairs,
                                 args.oracle_pairs, args.warmup, args.steps)
    line = {"metric": METRIC + "; learned-init vs plain", "workload": "learned-init vs plain",
            "value": res["learned"]["pairs_per_s"], "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (network bf16)", "data": "synthetic (seeded kinematic Kikuchi generator)",
            "config": {"workload": res["workload"], "pairs": args.pairs}, "learned_vs_plain": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ comparison methods (Fig. 2-3 analogue)
def run_compare(args, rank, world, local_rank):
    """Test-set-1 analogue of Section 3.1: in-plane rotations of 1..10 degrees about the
    detector normal, several reference orientations per angle, noise-free 256x256 patterns,
    demons 4 levels x 50 iterations with sigma = 1 smoothing, 25 ROIs of 64x64.  (The paper
    runs 25 iterations without smoothing on dense dynamical simulations; on the sparse
    kinematic patterns here the unsmoothed field diverges, so the workloads' smoothing is
    kept.)  Reports the rotation error of the four methods of Fig. 2 and the MAE / PH /
    SSIM of Fig. 3, and the throughput of the whole comparison."""
    import numpy as np
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as SG
    from synth import kikuchi as K
    torch.cuda.set_device(local_rank)
    H = 256
    angles = list(range(1, 11))
    n_ori = args.compare_orientations
    geom = K.Geometry()
    gs, Fs, keys = [], [], []
    for a in angles:
        for o in range(n_ori):
            gs.append(K.random_rotation(1907, o))
            Fs.append(K.axis_angle([0.0, 0.0, 1.0], np.radians(a)))
            keys.append(0)
    B = len(gs)
    tests = SG.render_batch(gs, Fs, keys, H, H, geom, 500.0, noise=False)
    refs = SG.render_batch(gs, [np.eye(3)] * B, keys, H, H, geom, 500.0, noise=False)
    ridx = torch.arange(B, dtype=torch.int32, device="cuda")
    roi = K.roi_grid(H, H, 64, False)
    pipe = Pipeline(PipelineConfig(H, H, roi, 64, 4, (50, 50, 50, 50), 1.0, 1.0))
    out = {}
    for _ in range(args.warmup):
        pipe.compare(refs, tests, ridx, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pipe.compare(refs, tests, ridx, out=out)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3

    def polar(F):
        U, _, Vt = np.linalg.svd(F)
        return U @ Vt

    def rot_err(A, Bm):
        return float(np.arccos(np.clip((np.trace(A.T @ Bm) - 1) / 2, -1, 1)))
    res = []
    for i, a in enumerate(angles):
        sl = slice(i * n_ori, (i + 1) * n_ori)
        row = {"angle_deg": a}
        for m in "abcd":
            Fm = out[f"F_{m}"].cpu().numpy().reshape(-1, 3, 3)[sl]
            row[f"rot_err_{m}_rad"] = float(np.mean([rot_err(polar(f), Ft) for f, Ft in zip(Fm, Fs[sl])]))
            row[f"mae_{m}_rad"] = float(out[f"mae_{m}"].cpu().numpy()[sl].mean())
        for m in "acd":
            row[f"ph_{m}"] = float(out[f"phm_{m}"].cpu().numpy()[sl].mean())
        row["ssim_b"] = float(out["ssim_b"].cpu().numpy()[sl].mean())
        row["ssim_no_warp"] = float(out["ssim_none"].cpu().numpy()[sl].mean())
        res.append(row)
    line = {"metric": "comparison methods of Fig. 2-3 (a: XCF, b: demons, c: XCF remap + XCF, d: demons remap + XCF)",
            "workload": "compare", "value": B * args.steps / t, "unit": "pairs/s (all four methods and metrics)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic (seeded kinematic Kikuchi generator), noise-free",
            "config": {"workload": f"in-plane rotations 1..10 deg about the detector normal, {n_ori} reference "
                                   f"orientations each, 256x256, demons 4 levels x 50 it, sigma 1, 25 ROIs 64x64"},
            "per_angle": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pipe.close()
    return 0


# ------------------------------------------------------------------ single pair (latency)
def single_pair_latency(local_rank, warmup=3, reps=20):
    """Latency of one pair through the whole chain (128x128, 3 levels x 50 iterations, 21 ROIs 32x32),
    with the per-level CUDA graphs and with direct launches: {graphs: (ms, launches per pair)}."""
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import kikuchi as K
    torch.cuda.set_device(local_rank)
    spec = K.config1()
    refs, tests, ridx, _ = K.make_scan(spec)
    refs, tests, ridx = (torch.from_numpy(refs).cuda(), torch.from_numpy(tests).cuda(), torch.from_numpy(ridx).cuda())
    roi = K.roi_grid(128, 128, 32, True)
    res = {}
    for graphs in (1, 0):
        pipe = Pipeline(PipelineConfig(128, 128, roi, 32, 3, (50, 50, 50)))
        P.hrebsd_set_option(pipe.ctx, P.OPT_GRAPHS, graphs)
        out = {}
        for _ in range(max(3, warmup)):
            pipe.run(refs, tests, ridx, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = P.hrebsd_launch_count(pipe.ctx)
        e0.record()
        for _ in range(reps):
            pipe.run(refs, tests, ridx, out=out)
        e1.record()
        torch.cuda.synchronize()
        res[graphs] = (e0.elapsed_time(e1) / reps, (P.hrebsd_launch_count(pipe.ctx) - l0) / reps)
        pipe.close()
    return res


def run_single(args, rank, world, local_rank):
    """The single-pair workload (128x128, 3 levels x 50 iterations, 21 ROIs 32x32): latency of one
    pair through the whole chain, with the per-level CUDA graphs and with direct launches."""
    reps = max(20, args.steps)
    res = single_pair_latency(local_rank, args.warmup, reps)
    line = {"metric": "single-pair latency (demons+XCF)", "workload": "single", "value": res[1][0], "unit": "ms/pair",
            "higher_is_better": False, "n_gpus": 1, "steps": reps, "warmup": max(3, args.warmup),
            "data": "synthetic (seeded kinematic Kikuchi generator)", "dtype": "f32",
            "config": {"workload": "1 pair 128x128, 2 deg, 3 levels x 50 iterations, 21 ROIs 32x32"},
            "ms_per_pair_graphs": res[1][0], "ms_per_pair_direct": res[0][0], "kernel_launches_per_pair": res[1][1]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ learned initialiser alone (a10)
def run_cnn(args, rank, world, local_rank):
    """U-Net inference of the learned initialiser alone: --pairs pairs of 64x64 (reference, test)
    BF16 inputs, He-normal weights; forward on the tcgen05 convolutions (the default) and on the
    mma.sync kernels.  The timed region is device work only (inputs resident)."""
    import torch
    import paper_1907_05993_gb300 as P
    from paper_1907_05993_gb300 import learned as LN
    torch.cuda.set_device(local_rank)
    B = args.pairs
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn((B, 2, 64, 64), device="cuda", generator=g).to(torch.bfloat16)
    out = torch.empty((B, 2, 64, 64), device="cuda")
    # 2 x MACs per pair: 3x3 layers (input channels padded to 16) + the 1x1 head
    layers = [(16, 16, 64), (16, 16, 64), (16, 32, 32), (32, 32, 32), (32, 64, 16), (64, 64, 16), (64, 128, 8),
              (128, 128, 8), (192, 64, 16), (64, 64, 16), (96, 32, 32), (32, 32, 32), (48, 16, 64), (16, 16, 64)]
    flop = sum(2 * 9 * ci * co * r * r for ci, co, r in layers) + 2 * 16 * 2 * 64 * 64
    res = {}
    for tc in (1, 0):
        ctx = P.hrebsd_create(local_rank)
        P.hrebsd_set_option(ctx, P.OPT_CNN_TC, tc)
        P.hrebsd_cnn_init(ctx, LN.init_params(0))
        for _ in range(max(3, args.warmup)):
            P.hrebsd_cnn_infer(ctx, x, B, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = P.hrebsd_launch_count(ctx)
        e0.record()
        for _ in range(args.steps):
            P.hrebsd_cnn_infer(ctx, x, B, out)
        e1.record()
        torch.cuda.synchronize()
        P.hrebsd_device_error(ctx)
        ms = e0.elapsed_time(e1) / args.steps
        res[tc] = (ms, (P.hrebsd_launch_count(ctx) - l0) / args.steps)
        # one training step (forward, MSE loss, backward, Adam) on a batch of 256 pairs
        TB = 256
        tgt = torch.randn((TB, 2, 64, 64), device="cuda", generator=g) * 0.5
        loss = torch.zeros(1, device="cuda")
        for _ in range(max(3, args.warmup)):
            P.hrebsd_cnn_train_step(ctx, x[:TB], tgt, TB, 1e-4, loss)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            P.hrebsd_cnn_train_step(ctx, x[:TB], tgt, TB, 1e-4, loss)
        e1.record()
        torch.cuda.synchronize()
        P.hrebsd_device_error(ctx)
        res[("train", tc)] = e0.elapsed_time(e1) / args.steps
        P.hrebsd_destroy(ctx)
    line = {"metric": "learned-initialiser inference pairs/s", "workload": "cnn", "value": B / (res[1][0] / 1e3),
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "higher_is_better": True,
            "data": "synthetic (random BF16 inputs, He-normal weights)", "dtype": "bf16 (FP32 accumulation)",
            "config": {"workload": f"U-Net 16-32-64-128 inference, {B} pairs of 64x64",
                       "gflop_per_pair": flop / 1e9},
            "ms_per_step": res[1][0], "tflops": flop * B / (res[1][0] / 1e3) / 1e12, "gpu_launches": res[1][1],
            "mma_sync": {"ms_per_step": res[0][0], "pairs_per_s": B / (res[0][0] / 1e3),
                         "tflops": flop * B / (res[0][0] / 1e3) / 1e12},
            "train_step": {"batch": 256, "ms_tcgen05": res[("train", 1)], "ms_mma_sync": res[("train", 0)],
                           "pairs_per_s": 256 / (res[("train", 1)] / 1e3),
                           "note": "forward, loss, backward, Adam; first column: forward, weight-gradient and (11 of 13 "
                                   "layers) input-gradient convolutions on tcgen05"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ large patterns (f4)
def run_large(args, rank, world, local_rank):
    """Patterns at the paper's scale (Section 3.1): 1244 x 1024, 7 pyramid levels (widths 1244, 622, 311,
    155, 77, 38, 19), 20 iterations per level (the paper's Inconel settings), 100 ROIs of 256 x 256 on a
    10 x 10 grid."""
    import numpy as np
    import torch
    from paper_1907_05993_gb300.pipeline import Pipeline, PipelineConfig
    from synth import gpu as SG
    from synth import kikuchi as K
    torch.cuda.set_device(local_rank)
    n = args.large_pairs
    H, W = 1024, 1244
    spec = K.ScanSpec(n_pairs=n, H=H, W=W, n_refs=4, mis_lo_deg=0.0, mis_hi_deg=6.0, strain=5e-4,
                      strain_mode="sigma", counts=500.0, seed=6)
    refs, tests, ridx, _ = SG.make_scan_gpu(spec)
    roi = K.roi_grid_n(H, W, 256, 10)
    pipe = Pipeline(PipelineConfig(H, W, roi, 256, 7, (20,) * 7))
    out = {}
    for _ in range(args.warmup):
        pipe.run(refs, tests, ridx, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pipe.run(refs, tests, ridx, out=out)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    line = {"metric": "pattern pairs/s (demons+XCF), large patterns", "workload": "large", "value": n * args.steps / t,
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic (seeded kinematic Kikuchi generator)", "dtype": "f32",
            "config": {"workload": f"{n} pairs of 1244x1024, 4 references, mis U(0,6) deg, 7 levels x 20 iterations, "
                                   f"100 ROIs 256x256", "ms_per_pair": 1e3 * t / (n * args.steps)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pipe.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--pairs", type=int, default=10_000)
    ap.add_argument("--cpu-sample", type=int, default=48)
    ap.add_argument("--ref-sample", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("scan", "learned", "compare", "large", "single", "cnn"),
                    default="scan")
    ap.add_argument("--large-pairs", type=int, default=256)
    ap.add_argument("--compare-orientations", type=int, default=16)
    ap.add_argument("--train-pairs", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--learned-start", type=int, default=64, choices=(64, 128))
    ap.add_argument("--oracle-pairs", type=int, default=500)
    ap.add_argument("--no-learned", action="store_true", help="default run: skip the learned-vs-plain comparison")
    ap.add_argument("--no-single", action="store_true", help="default run: skip the single-pair latency")
    ap.add_argument("--lvp-train-pairs", type=int, default=20_000)
    ap.add_argument("--lvp-epochs", type=int, default=20)
    ap.add_argument("--learned-caps", type=int, nargs=4, default=(25, 25, 10, 0))
    ap.add_argument("--tile-variants", type=int, nargs=4, default=None,
                    help="scan workload: demons tile shape per level, finest first (no autotuning)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "learned":
        return run_learned(args, rank, world, local_rank)
    if args.workload == "compare":
        return run_compare(args, rank, world, local_rank)
    if args.workload == "large":
        return run_large(args, rank, world, local_rank)
    if args.workload == "single":
        return run_single(args, rank, world, local_rank)
    if args.workload == "cnn":
        return run_cnn(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
