#!/usr/bin/env python3
"""Throughput and latency of the PIV correction path on GB300.

Workload: 1024 x 1024 12-bit (uint16) synthetic particle pairs, 0.03 ppp,
d_p U(2, 4) px, 10 % out-of-plane loss, uniform 12 px + shear layer + Lamb-Oseen
vortex; 2-level correlation pyramid, then passes of 64 -> 32 -> 16 px windows at
50 % overlap with a +-4 px search (127 x 127 vectors per pair).  One step = one
batch of 64 pairs through the whole path (pyramid, deformation, correlation,
peak, Gaussian fit, outlier test, interpolation, vorticity), inputs resident
in device memory (256 MiB per step, larger than L2).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import datetime
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1 MP PIV pairs/s and p99 latency, BF16 vs FP32 path at ≤0.01 px error vs oracle"
N_DISTINCT = 8          # distinct synthetic pairs, replicated to fill a batch
BATCH = 64
WORKLOAD_R1 = ("paper_1mp_16px_r1: the 1 MP pair below with the paper's own operating point: 2-level pyramid, "
               "32 px (+-4) -> 16 px at 50% with a +-1 stencil search; 127x127 vectors")
WORKLOAD = ("paper_1mp_u16: 1024x1024 uint16 (12-bit) pair, 0.03 ppp, d_p U(2,4), 10% particle loss, "
            "uniform 12 px + tanh shear + Lamb-Oseen; 2-level pyramid, passes 64->32->16 px, 50% overlap, "
            "search +-4; 127x127 vectors")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=BATCH)
    p.add_argument("--precisions", default="fp32,bf16,fp16")
    p.add_argument("--headline", default="fp32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--latency-requests", type=int, default=200)
    p.add_argument("--workload", default="paper_1mp", choices=["paper_1mp", "paper_1mp_r1"],
                   help="paper_1mp_r1: the paper's 16 px / +-1 operating point on the same images")
    p.add_argument("--mode", default="full",
                   choices=["full", "ncu", "serve", "precision", "adjoint", "sizes", "preprocess", "tcrate"],
                   help="ncu: one warm-up step and one step of the headline path, nothing else (profiler runs); "
                        "serve: the streaming mix (Poisson arrivals over camera streams); "
                        "precision: the 8 MP Fourier-mode pair, FP32/BF16/FP16 fields against the FP64 oracle")
    p.add_argument("--requests", type=int, default=10000)
    p.add_argument("--streams", type=int, default=32)
    p.add_argument("--load", type=float, default=0.7, help="Poisson rate as a fraction of the saturation rate")
    p.add_argument("--extra-loads", default="0.5", help="further load fractions reported beside --load (serve mode)")
    p.add_argument("--serve-precision", default="fp32", choices=["fp32", "bf16", "fp16"],
                   help="correlation precision of the serving mix")
    p.add_argument("--serve-compare", default="", help="further precisions measured in the serving mix, e.g. bf16")
    p.add_argument("--slots", type=int, default=8, help="concurrent batches (CUDA streams) in the serving mix")
    p.add_argument("--repeats", type=int, default=3, help="Poisson runs at --load with fresh arrival seeds")
    p.add_argument("--upload", default="engine", choices=["engine", "executor"],
                   help="serve mode: pinned host frames read by the engine's upload kernel, or copied to the "
                        "device by the executor (one copy call per image)")
    return p.parse_args()


# ------------------------------------------------------- replica timing --

def replica_seeds(rank: int, n: int):
    """Seeds of the distinct pairs a replica renders: disjoint across ranks."""
    return [1002 + 100 * rank + k for k in range(n)]


def timed_replicas(step, steps: int, warmup: int, barrier, start_timer, reduce_max) -> float:
    """Warm-up steps, then `steps` timed steps bracketed by a barrier on both
    sides; returns the slowest rank's elapsed milliseconds.  start_timer()
    returns a function giving the elapsed milliseconds since it was called
    (CUDA events on the launching stream on the GPU)."""
    for _ in range(warmup):
        step()
    barrier()
    stop = start_timer()
    for _ in range(steps):
        step()
    ms = stop()
    barrier()
    return reduce_max(ms)


def aggregate_rate(world: int, units_per_rank_step: int, steps: int, max_ms: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank_step * steps / (max_ms / 1000.0)


# ------------------------------------------------------------ CPU oracle --

def _oracle_pair(job):
    """Render one pair and run the FP64 oracle on it; returns timing and field.
    job: a seed, or (seed, workload name)."""
    import numpy as np  # noqa: F401
    import oracle
    from synth import workloads as wl
    seed, name = (job, "paper_1mp") if isinstance(job, int) else job
    w = wl.paper_1mp(seed=seed)
    A, B = w.render()
    sc = (wl.paper_1mp_r1(seed=seed) if name == "paper_1mp_r1" else w).schedule
    t0 = time.perf_counter()
    r = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    dt = time.perf_counter() - t0
    return seed, dt, r.u, r.v


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_round(pool, seeds):
    """Runs the oracle on one pair per worker; the round lasts as long as its
    slowest pair (rendering and process overhead excluded)."""
    res = pool.map(_oracle_pair, seeds, chunksize=1)
    return max(r[1] for r in res), res


def _render_stream(args):
    """Frames of one camera stream: a ring of pairs whose vortex advects 0.5 px/frame."""
    import synth
    from synth import workloads as wl
    stream, W, H, bits, ring = args
    out = []
    for f in range(ring):
        flow = wl.serving_stream_flow(stream, f, W, H)
        spec = synth.ImageSpec(W=W, H=H, bit_depth=bits, ppp=0.05, dp=(2.5, 2.5), seed=50000 + 131 * stream + f)
        out.append(synth.render_pair(spec, flow))
    return stream, out


def run_serve(args):
    """Streaming mix: camera streams of 512^2 .. 3840x2160, u8 or 12-bit,
    previous field as predictor, at most 64 pairs per launch, 40 GB admission
    budget; saturation throughput, then Poisson arrivals at a fraction of it
    with p50/p99 latency, repeated with fresh arrival seeds.  The mix runs in
    the faster correlation precision (FP32) unless told otherwise; further
    precisions are measured the same way and reported beside it."""
    import synth
    from synth import workloads as wl
    ring = 4
    slots = args.slots
    rnd = synth.uniform(777, 2 * args.streams)
    cum = np.cumsum([w for _, _, w in wl.SERVING_SIZES])
    streams = []
    for s in range(args.streams):
        k = int(np.searchsorted(cum, rnd[2 * s] * cum[-1], side="right"))
        W, H, _ = wl.SERVING_SIZES[min(k, len(wl.SERVING_SIZES) - 1)]
        bits = 8 if rnd[2 * s + 1] < 0.5 else 12
        streams.append((s, W, H, bits, ring))
    with mp.get_context("spawn").Pool(min(_host_cores(), len(streams))) as pool:
        frames = dict(pool.map(_render_stream, streams))
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    from paper_2504_17987_gb300 import serving as sv
    torch.cuda.set_device(0)
    pinned = {s: [(rp.to_device(a, pin=True), rp.to_device(b, pin=True)) for a, b in frames[s]] for s in frames}

    def requests(n, rate, seed):
        arr = wl.poisson_arrivals(n, rate, seed) if rate > 0 else [0.0] * n
        out = []
        for k in range(n):
            s = k % args.streams
            f = k // args.streams
            _, W, H, bits, _ = streams[s]
            out.append(sv.Request(rid=k, stream=s, frame=f, arrival=arr[k], key=(W, H, bits),
                                  payload=pinned[s][f % ring]))
        return out

    def scheduler(ex):
        return sv.Scheduler(ex, max_batch=64, slots=slots, hbm_budget=40e9)

    def summary(sch, rep):
        wait = [1000.0 * (r.dispatched - r.arrival) for r in sch.done]
        service = [1000.0 * (r.done - r.dispatched) for r in sch.done]
        return {"pairs_per_s": rep["pairs_per_s"], "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
                "max_ms": rep["max_ms"], "mean_batch": rep["mean_batch"],
                "queue_p50_ms": float(np.percentile(wait, 50)), "queue_p99_ms": float(np.percentile(wait, 99)),
                "service_p50_ms": float(np.percentile(service, 50)),
                "service_p99_ms": float(np.percentile(service, 99)),
                "host_busy_frac": rep["host_busy_frac"], "host_us_per_batch": rep["host_us_per_batch"]}

    def measure(precision, repeats):
        ex = sv.GpuExecutor(slots=slots, precision=precision, max_batch=64, cold_batch=8, prewarm=True,
                            host_frames=args.upload == "engine")
        # every engine (frame size, mode, slot) and every batch size's graph exist before any timing
        for key in sorted({(W, H, bits) for _, W, H, bits, _ in streams}):
            for mode in (sv.COLD, sv.WARM):
                for slot in range(slots):
                    ex._engine(key, mode, slot)
        torch.cuda.synchronize()
        # saturation: every request available at once (also warms engines and graphs)
        n_sat = min(args.requests, 2000)
        sat_s = scheduler(ex)
        sat = sat_s.run(requests(n_sat, 0.0, 1), realtime=False)
        rate = args.load * sat["pairs_per_s"]
        torch.cuda.synchronize()
        runs = []
        for rep_i in range(repeats):
            sch = scheduler(ex)
            rep = sch.run(requests(args.requests, rate, 2 + rep_i))
            runs.append((sch, rep))
        others = {}
        for frac in [float(x) for x in args.extra_loads.split(",") if x.strip()]:
            sch = scheduler(ex)
            r2 = sch.run(requests(args.requests, frac * sat["pairs_per_s"], 100 + int(100 * frac)))
            others[str(frac)] = dict(summary(sch, r2), arrival_rate_per_s=frac * sat["pairs_per_s"])
        ex.close()
        return sat, rate, runs, others

    sat, rate, runs, others = measure(args.serve_precision, max(1, args.repeats))
    # the run with the median p99 is the headline; every run is listed
    order = sorted(range(len(runs)), key=lambda i: runs[i][1]["p99_ms"])
    sch, rep = runs[order[len(order) // 2]]
    by_size = {}
    for r in sch.done:
        by_size.setdefault(f"{r.key[0]}x{r.key[1]}", []).append(1000.0 * r.latency)
    per_size = {k: {"n": len(v), "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
                for k, v in sorted(by_size.items())}
    steady = sorted(1000.0 * r.latency for r in sch.done if r.frame >= 3 and r.error is None)
    steady_p = {"p50_ms": float(np.percentile(steady, 50)), "p99_ms": float(np.percentile(steady, 99)),
                "what": "requests after each stream's first three frames (start-up transient excluded)"}
    s = summary(sch, rep)
    split = {k: s[k] for k in ("queue_p50_ms", "queue_p99_ms", "service_p50_ms", "service_p99_ms")}
    p99s = [r[1]["p99_ms"] for r in runs]
    compare = {}
    for prec in [x.strip() for x in args.serve_compare.split(",") if x.strip() and x.strip() != args.serve_precision]:
        sat2, rate2, runs2, _ = measure(prec, 1)
        compare[prec] = dict(summary(*runs2[0]), saturation_pairs_per_s=sat2["pairs_per_s"],
                             saturation_mean_batch=sat2["mean_batch"], arrival_rate_per_s=rate2)
    mp_per_pair = sum(W * H for _, W, H, _, _ in streams) / len(streams) / 1e6
    line = {"mode": "serve", "metric": "streaming mix p50/p99 latency and pairs/s", "unit": "pairs/s",
            "value": rep["pairs_per_s"], "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "max_ms": rep["max_ms"],
            "requests": rep["requests"], "dropped": rep["dropped"], "mean_batch": rep["mean_batch"],
            "host_busy_frac": rep["host_busy_frac"], "host_us_per_batch": rep["host_us_per_batch"],
            "arrival_rate_per_s": rate, "saturation_pairs_per_s": sat["pairs_per_s"],
            "saturation_mean_batch": sat["mean_batch"], "saturation_host_busy_frac": sat["host_busy_frac"],
            "mean_megapixels_per_pair": mp_per_pair,
            "p99_ms_per_run": p99s, "p99_spread": max(p99s) / max(1e-9, min(p99s)),
            "runs": [summary(*r) for r in runs],
            "latency_by_frame_size": per_size, "latency_split": split, "steady_state": steady_p,
            "other_loads": others, "other_precisions": compare,
            "config": {"streams": args.streams, "sizes": wl.SERVING_SIZES, "precision": args.serve_precision,
                       "slots": slots, "max_pairs_per_launch": 64, "max_megapixels_per_launch": 16,
                       "hbm_budget_gb": 40, "ring_frames_per_stream": ring, "graphs_prewarmed": True,
                       "repeats": len(runs), "upload": args.upload},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    synth.build()
    cores = _host_cores()
    per_step = cores
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_round(pool, [1002 + k for k in range(per_step)])
        times = []
        for _ in range(args.steps):
            dt, _ = oracle_round(pool, [1002 + k for k in range(per_step)])
            times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} pairs per step (one per core), {args.steps} steps"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- precision case --

def _oracle_8mp(seed: int):
    import oracle
    from synth import workloads as wl
    w = wl.fourier_8mp(seed=seed)
    A, B = w.render()
    sc = w.schedule
    t0 = time.perf_counter()
    r = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    return time.perf_counter() - t0, r.u, r.v, r.vort, r.mask


def run_precision(args):
    """8 MP pair (3840x2160 u8, 8 Fourier modes, 48 -> 24 px, +-6, 2-level
    pyramid): per-field error of each precision against the FP64 oracle, and
    each precision's throughput at batch 8."""
    import numpy as np
    pool = mp.get_context("spawn").Pool(1)
    pending = pool.apply_async(_oracle_8mp, (1004,))
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    from synth import workloads as wl
    wk = wl.fourier_8mp(seed=1004)
    A, B = wk.render()
    H, W = A.shape
    a, b = rp.to_device(A), rp.to_device(B)
    out = {}
    fields = {}
    for prec in ("fp32", "bf16", "fp16"):
        cfg = rp.Config.from_schedule(W, H, wk.schedule, bit_depth=8, precision=prec, max_batch=8)
        eng = rp.Engine(cfg)
        res = eng.process_pair(a, b)
        torch.cuda.synchronize()
        fields[prec] = [t.cpu().numpy().astype(np.float64) for t in res]
        outs = eng.empty_outputs(8)
        for _ in range(3):
            eng.process_batch([a] * 8, [b] * 8, outs=outs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            eng.process_batch([a] * 8, [b] * 8, outs=outs)
        e1.record()
        torch.cuda.synchronize()
        out[prec] = {"pairs_per_s": 40 / (e0.elapsed_time(e1) / 1000.0)}
        eng.close()
    dt, ou, ov, oom, omask = pending.get()
    pool.close()

    def stats(d):
        d = np.abs(d)
        return {"p50": float(np.median(d)), "p99": float(np.percentile(d, 99)), "max": float(d.max()),
                "rms": float(np.sqrt(np.mean(d * d)))}
    for prec, (u, v, om, m) in fields.items():
        out[prec]["err_vs_oracle"] = {"u_px": stats(u - ou), "v_px": stats(v - ov), "vort_per_frame": stats(om - oom),
                                      "mask_agreement": float(np.mean(m == omask))}
    line = {"mode": "precision", "workload": "fourier_8mp_u8: 3840x2160 u8, 0.05 ppp, d_p 2.5, 8 Fourier modes "
            "(max 16 px); 2-level pyramid, 48 -> 24 px at 50 %, search +-6; 319x179 vectors",
            "oracle_s": dt, "paths": out, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------- pre-processing --

def run_preprocess(args):
    """High-pass (15 x 15 box) and CLAHE (8 x 8 tiles, clip 2) of both frames of
    a 1 MP 12-bit pair, then the correction path on the float frames: time per
    pair of each."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    from synth import workloads as wl
    wk = wl.paper_1mp()
    A, B = wk.render()
    H, W = A.shape
    a, b = rp.to_device(A), rp.to_device(B)

    # outputs and scratch made once, so that the timed loop holds the kernels
    # and their launches, not allocations
    from paper_2504_17987_gb300 import binding
    outs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(2)]
    scr = [torch.empty(binding.preprocess_scratch_bytes(W, H, (8, 8)), dtype=torch.uint8, device="cuda")
           for _ in range(2)]

    def pre():
        return (rp.stage_preprocess(a, 4095, hp=7, tiles=(8, 8), clip_pct=200, out=outs[0], scratch=scr[0]),
                rp.stage_preprocess(b, 4095, hp=7, tiles=(8, 8), clip_pct=200, out=outs[1], scratch=scr[1]))
    for _ in range(3):
        pa, pb = pre()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        pa, pb = pre()
    e1.record()
    torch.cuda.synchronize()
    pre_ms = e0.elapsed_time(e1) / 20
    cfg = rp.Config.from_schedule(W, H, wk.schedule, bit_depth=12, float_frames=True, max_batch=1)
    eng = rp.Engine(cfg)
    for _ in range(3):
        eng.process_pair(pa, pb)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        eng.process_pair(pa, pb)
    e1.record()
    torch.cuda.synchronize()
    path_ms = e0.elapsed_time(e1) / 20
    eng.close()
    # temporal smoothing of a field of 64 Mi floats (> L2): x and the state read, the state written
    n_ema = 1 << 26
    x = torch.rand(n_ema, device="cuda")
    st = torch.rand(n_ema, device="cuda")
    for _ in range(3):
        rp.stage_ema(x, st, 0.5)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        rp.stage_ema(x, st, 0.5)
    e1.record()
    torch.cuda.synchronize()
    ema_ms = e0.elapsed_time(e1) / 20
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    pre_b = 2 * W * H * (2 + 4)  # both frames: u16 in, float out
    ema_b = 12 * n_ema
    print(json.dumps({"mode": "preprocess", "workload": WORKLOAD, "preprocess_ms_per_pair": pre_ms,
                      "path_ms_per_pair_float_frames": path_ms, "ema_ms_64mi": ema_ms,
                      "roofline": {"peak_gbs": hbm,
                                   "preprocess": {"algorithmic_bytes": pre_b, "gbs": pre_b / (pre_ms * 1e-3) / 1e9,
                                                  "frac": pre_b / (pre_ms * 1e-3) / 1e9 / hbm,
                                                  "what": "u16 frames in, float frames out (one pair; launch- and "
                                                          "latency-bound at this size)"},
                                   "ema": {"algorithmic_bytes": ema_b, "gbs": ema_b / (ema_ms * 1e-3) / 1e9,
                                           "frac": ema_b / (ema_ms * 1e-3) / 1e9 / hbm,
                                           "what": "x and state read, state written, 64 Mi floats"}},
                      "data": "synthetic"}), flush=True)
    return 0


# ------------------------------------------------------------ size sweep --

SWEEP_SIZES = [(512, 512), (768, 640), (1024, 1024), (1600, 1200), (2048, 2048), (3840, 2160), (4096, 4096),
               (8192, 4096)]


def run_sizes(args):
    """Frames per second against image size (0.26 .. 33.6 MP) for the paper's
    16 px / 50 % operating point (pyramid, 32 px +-4, then 16 px +-1), the
    shape of the paper's throughput-against-size figure (Sec. 4.1).  Batches
    hold about 64 MP."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    from synth import workloads as wl
    sched = wl.paper_1mp_r1().schedule
    rows = []
    for (W, H) in SWEEP_SIZES:
        wk = wl.paper_1mp(seed=1002, W=W, H=H)
        A, B = wk.render()
        a, b = rp.to_device(A), rp.to_device(B)
        n = max(1, min(64, int(64e6 // (W * H))))
        cfg = rp.Config.from_schedule(W, H, sched, bit_depth=12, precision=args.headline, max_batch=n)
        eng = rp.Engine(cfg)
        outs = eng.empty_outputs(n)
        if n == 1:
            outs = tuple(o.unsqueeze(0) for o in outs)
        for _ in range(3):
            eng.process_batch([a] * n, [b] * n, outs=outs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        steps = 10
        for _ in range(steps):
            eng.process_batch([a] * n, [b] * n, outs=outs)
        e1.record()
        torch.cuda.synchronize()
        fps = n * steps / (e0.elapsed_time(e1) / 1000.0)
        rows.append({"width": W, "height": H, "megapixels": W * H / 1e6, "batch": n, "pairs_per_s": fps,
                     "megapixels_per_s": fps * W * H / 1e6, "vectors": eng.nx * eng.ny})
        eng.close()
        del a, b, outs
        torch.cuda.empty_cache()
    print(json.dumps({"mode": "sizes", "precision": args.headline, "workload": WORKLOAD_R1, "rows": rows,
                      "data": "synthetic"}), flush=True)
    return 0


def run_tc_rate(args):
    """Cycles per tcgen05.mma (kind::f16, K = 16) against M and N, from one
    thread issuing 256 MMAs back to back (libtcrate); with the clock sampled,
    the tensor-core rate each shape reaches."""
    import ctypes

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_17987_gb300 import build as b
    lib = ctypes.CDLL(b.build_tc_rate())
    lib.tc_rate_cycles.restype = ctypes.c_double
    lib.tc_rate_cycles.argtypes = [ctypes.c_int] * 4
    torch.cuda.init()
    rows = []
    for M, N, nacc in [(128, 16, 1), (128, 16, 8), (64, 16, 8), (128, 32, 8), (128, 64, 8), (128, 128, 4),
                       (128, 256, 1), (128, 256, 2)]:
        cyc = lib.tc_rate_cycles(M, N, 256, nacc)
        if cyc < 0 or cyc >= 1e9:
            raise RuntimeError(f"tc_rate_cycles({M}, {N}) failed: {cyc}")
        rows.append({"M": M, "N": N, "K": 16, "accumulators": nacc, "cycles_per_mma": round(cyc, 1),
                     "mac_per_cycle": round(M * N * 16 / cyc, 1)})
    # several issuing CTAs per SM (64 KB of shared memory each: at most three
    # per SM): is the cost per MMA the issuer's or the SM's?
    lib.tc_rate_sm.restype = ctypes.c_double
    lib.tc_rate_sm.argtypes = [ctypes.c_int] * 7 + [ctypes.POINTER(ctypes.c_double)]
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def sm_rate(M, N, nacc, issuers, ctas, cols):
        pc = ctypes.c_double()
        cyc = lib.tc_rate_sm(M, N, 256, nacc, issuers, ctas, cols, ctypes.byref(pc))
        if cyc < 0 or cyc >= 1e9:
            raise RuntimeError(f"tc_rate_sm({M}, {N}, {issuers} issuers, {ctas} CTAs) failed: {cyc}")
        return {"M": M, "N": N, "K": 16, "issuers_per_cta": issuers, "sm_cycles_per_mma": round(cyc, 1),
                "cta_cycles_per_mma": round(pc.value, 1), "sm_mac_per_cycle": round(M * N * 16 / cyc, 1)}

    per_sm = [dict(sm_rate(M, N, nacc, 1, k * sms, 128), ctas_per_sm=k)
              for M, N, nacc in [(128, 16, 8), (128, 128, 1)] for k in (1, 2, 3)]
    # several issuing warps in one CTA (one CTA on one SM)
    per_warp = [sm_rate(M, N, nacc, k, 1, 512) for M, N, nacc in [(128, 16, 8), (128, 64, 2)] for k in (1, 2, 4)]
    print(json.dumps({"mode": "tcrate", "rows": rows, "several_ctas_per_sm": per_sm,
                      "several_issuers_per_cta": per_warp}), flush=True)
    return 0


# ------------------------------------------------------ differentiation --

def run_adjoint(args):
    """Score and gradient through the warp at 1 MP (u8, 32 px at 75 %, 125x125
    nodes): time of rpiv_backward, and the 5-step gradient refinement."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    import synth
    from synth import workloads as wl
    wk = wl.diff_1mp()
    A, B = wk.render()
    H, W = A.shape
    cfg = rp.Config(W, H, windows=(32,), overlaps=(0.75,), radii=(8,), bit_depth=8)
    eng = rp.Engine(cfg)
    a, b = rp.to_device(A), rp.to_device(B)
    X, Y = np.meshgrid(np.arange(125) * 8 + 15.5, np.arange(125) * 8 + 15.5)
    tu, tv = wk.flow.eval(X, Y)
    r = synth.uniform(3003, 2 * 125 * 125).reshape(2, 125, 125)
    u = torch.from_numpy((tu + 0.3 * (r[0] - 0.5)).astype(np.float32)).cuda()
    v = torch.from_numpy((tv + 0.3 * (r[1] - 0.5)).astype(np.float32)).cuda()
    for _ in range(3):
        eng.score_and_grad(a, b, u, v)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        eng.score_and_grad(a, b, u, v)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    rp.refine(eng, a, b, u, v, steps=5)  # first use: lazy module and allocator warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, hist = rp.refine(eng, a, b, u, v, steps=5)
    torch.cuda.synchronize()
    ref_ms = 1000 * (time.perf_counter() - t0)
    e_before = float(np.median(np.hypot(u.cpu().numpy() - tu, v.cpu().numpy() - tv)))
    # the adjoint must read both frames and the field, and write the gradient
    alg = 2 * W * H * 1 + 125 * 125 * 4 * 4
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = alg / (ms * 1e-3) / 1e9
    line = {"mode": "adjoint", "workload": "diff_1mp_u8: 1024x1024 u8, 32 px at 75 %, 125x125 nodes",
            "score_and_grad_ms": ms, "refine_5_steps_ms": ref_ms, "score_history": hist,
            "median_error_px_before": e_before,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg, "gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                         "what": "frames A, B (u8) and the field read, the gradient written, per call"},
            "data": "synthetic"}
    eng.close()
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- clocks --

def measure_fma_peak(index: int, reps: int = 30) -> dict:
    """The FP32 CUDA-core peak measured by the FMA-throughput microbenchmark
    (libfmapeak: 16 independent FMA chains per thread, 8 CTAs of 256 threads on
    every SM, as scalar FMAs and as packed fma.rn.f32x2 pairs), the shortest of
    `reps` launches of each, with the SM clock sampled while they run; the
    peak is the faster form.  Also the rate per SM and clock, to compare with
    the 128 FP32 lanes x 2 flop of the architecture."""
    import ctypes

    import torch

    from paper_2504_17987_gb300 import build as b
    lib = ctypes.CDLL(b.build_fma_peak())
    lib.fma_peak_run2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    st = torch.cuda.current_stream()
    forms = {}
    with ClockSampler(index) as cs:
        cs.mark_start()
        for packed in (0, 1):
            best, flops = ctypes.c_float(), ctypes.c_double()
            rc = lib.fma_peak_run2(8, 8192 if not packed else 4096, reps, packed, ctypes.byref(best),
                                   ctypes.byref(flops), ctypes.c_void_p(st.cuda_stream))
            if rc != 0:
                raise RuntimeError(f"FMA microbenchmark failed: CUDA error {rc}")
            forms["packed" if packed else "scalar"] = (best.value, flops.value)
        cs.mark_end()
    clk = cs.summary()
    sms = torch.cuda.get_device_properties(index).multi_processor_count
    rates = {k: f / (ms / 1e3) / 1e12 for k, (ms, f) in forms.items()}
    top = max(rates, key=rates.get)
    tflops = rates[top]
    mhz = (clk or {}).get("sm_mhz") or None
    per_clk = (tflops * 1e12 / (sms * mhz * 1e6)) if mhz else None
    return {"tflops": tflops, "form": top, "scalar_tflops": rates["scalar"], "packed_tflops": rates["packed"],
            "best_ms": forms[top][0], "flops_per_launch": forms[top][1], "sms": sms,
            "flop_per_sm_per_clock": per_clk, "clocks": clk}


class ClockSampler:
    """nvidia-smi samples every 20 ms around the timed region.  Sampling is
    live before the region starts (the first sample has arrived), and the
    summary keeps the samples whose timestamps fall between mark_start() and
    mark_end(); a region shorter than one interval falls back to the samples
    nearest to it, and says so."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.th = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            deadline = time.monotonic() + 10.0
            while not self.lines and self.proc.poll() is None and time.monotonic() < deadline:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        # one more interval, so that a sample taken at the very end is read
        time.sleep(2 * self.INTERVAL_MS / 1000.0)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.th is not None:
            self.th.join(timeout=2)

    @staticmethod
    def _stamp(text, arrived):
        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return arrived

    def _parse(self):
        rows = []
        for arrived, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = {nm for nm, val in zip(self.REASONS, parts[5:9]) if val.lower().startswith("active")}
            rows.append((self._stamp(parts[0], arrived), sm, mx, reasons))
        return rows

    def summary(self):
        rows = self._parse()
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "interval_ms": self.INTERVAL_MS}
        out = {"interval_ms": self.INTERVAL_MS}
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 <= r[0] <= self.t1]
            out["window_ms"] = round((self.t1 - self.t0) * 1000.0, 1)
            if not inside:
                before = [r for r in rows if r[0] < self.t0][-1:]
                after = [r for r in rows if r[0] > self.t1][:1]
                inside = before + after
                out["nearest_outside_region"] = True
            rows = inside
        out.update({"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                    "reasons": sorted(set().union(*(r[3] for r in rows))), "samples": len(rows)})
        return out


# ---------------------------------------------------------------- ours --

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "adjoint":
        return run_adjoint(args)
    if args.mode == "sizes":
        return run_sizes(args)
    if args.mode == "preprocess":
        return run_preprocess(args)
    if args.mode == "tcrate":
        return run_tc_rate(args)
    if args.mode == "serve":
        import numpy as np  # noqa: F811
        globals()["np"] = np
        return run_serve(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = _host_cores()
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_17987_gb300 as rp
    from synth import workloads as wl

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    B = args.batch
    seeds = replica_seeds(rank, N_DISTINCT)
    pairs = [wl.paper_1mp(seed=s).render() for s in seeds]
    sched = (wl.paper_1mp_r1() if args.workload == "paper_1mp_r1" else wl.paper_1mp()).schedule
    workload = WORKLOAD_R1 if args.workload == "paper_1mp_r1" else WORKLOAD
    H, W = pairs[0][0].shape
    a_dev = [rp.to_device(pairs[i % N_DISTINCT][0], dev) for i in range(B)]
    b_dev = [rp.to_device(pairs[i % N_DISTINCT][1], dev) for i in range(B)]
    in_bytes = sum(t.numel() * t.element_size() for t in a_dev + b_dev)

    if args.mode == "ncu":
        cfg = rp.Config.from_schedule(W, H, sched, bit_depth=12, precision=args.headline, max_batch=B)
        eng = rp.Engine(cfg, device=local)
        outs = eng.empty_outputs(B)
        for _ in range(2):
            eng.process_batch(a_dev, b_dev, outs=outs)
        torch.cuda.synchronize()
        eng.close()
        if pool is not None:
            pool.close()
        print(json.dumps({"mode": "ncu", "precision": args.headline, "batch": B, "steps": 2}))
        return 0

    precs = [p.strip() for p in args.precisions.split(",") if p.strip()]
    if args.headline not in precs:
        precs.append(args.headline)
    paths = {}
    traces = {}
    fields = {}
    clocks = None
    for prec in precs:
        cfg = rp.Config.from_schedule(W, H, sched, bit_depth=12, precision=prec, max_batch=B)
        eng = rp.Engine(cfg, device=local)
        outs = eng.empty_outputs(B)
        st = torch.cuda.current_stream()

        def start_timer():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)

            def stop():
                e1.record(st)
                e1.synchronize()
                return e0.elapsed_time(e1)
            return stop

        def step():
            eng.process_batch(a_dev, b_dev, outs=outs)

        for _ in range(args.warmup):
            step()
        with ClockSampler(local) as cs:
            cs.mark_start()
            ms = timed_replicas(step, args.steps, 0, barrier, start_timer, max_over_ranks)
            cs.mark_end()
        if prec == args.headline:
            clocks = cs.summary()
        fields[prec] = (outs[0][0].cpu().numpy(), outs[1][0].cpu().numpy())
        # stage trace (eager launches bracketed by events, same stream)
        eng.trace(True)
        for _ in range(3):
            eng.process_batch(a_dev, b_dev, outs=outs)
        recs = eng.trace_read()
        eng.trace(False)
        traces[prec] = recs
        paths[prec] = {"pairs_per_s": aggregate_rate(world, B, args.steps, ms), "ms_per_step": ms / args.steps,
                       "pass_ms_per_launch": {r["name"]: round(r["total_ms"] / r["launches"], 4)
                                              for r in recs if r["name"].startswith("pass/")}}
        eng.close()
        del outs
        torch.cuda.empty_cache()

    head = args.headline
    value = paths[head]["pairs_per_s"]

    # ---- end to end through the public API with pinned host buffers: each
    # step uploads its B pairs from pinned host memory (two copies, contiguous
    # frames), runs the path and downloads its fields; uploads go on a copy
    # stream into the other of two device input sets, so that step k + 1's
    # upload overlaps step k's compute, as a streaming caller would do it
    cfg = rp.Config.from_schedule(W, H, sched, bit_depth=12, precision=head, max_batch=B)
    eng = rp.Engine(cfg, device=local)
    a_host = torch.stack([rp.to_device(pairs[i % N_DISTINCT][0], pin=True) for i in range(B)]).pin_memory()
    b_host = torch.stack([rp.to_device(pairs[i % N_DISTINCT][1], pin=True) for i in range(B)]).pin_memory()
    a_in = [torch.empty_like(a_host, device=dev) for _ in range(2)]
    b_in = [torch.empty_like(b_host, device=dev) for _ in range(2)]
    outs = [eng.empty_outputs(B) for _ in range(2)]
    host_outs = [[torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs[0]] for _ in range(2)]
    out_bytes = sum(o.numel() * o.element_size() for o in outs[0])
    e2e_steps = max(30, args.steps)
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream(device=dev)
    uploaded = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    downloaded = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        j = k % 2
        with torch.cuda.stream(copy):
            copy.wait_event(computed[j])  # the set's previous batch has been consumed
            a_in[j].copy_(a_host, non_blocking=True)
            b_in[j].copy_(b_host, non_blocking=True)
            uploaded[j].record(copy)

    def run_steps(n):
        for j in range(2):
            computed[j].record(comp)
            downloaded[j].record(comp)
        upload(0)
        for k in range(n):
            j = k % 2
            comp.wait_event(uploaded[j])
            comp.wait_event(downloaded[j])  # the set's previous fields have reached the host
            eng.process_batch(list(a_in[j]), list(b_in[j]), outs=outs[j], stream=comp)
            computed[j].record(comp)
            if k + 1 < n:
                upload(k + 1)
            with torch.cuda.stream(copy):
                copy.wait_event(computed[j])
                for o, ho in zip(outs[j], host_outs[j]):
                    ho.copy_(o, non_blocking=True)
                downloaded[j].record(copy)
        copy.synchronize()
        comp.synchronize()

    run_steps(2)
    barrier()
    t0 = time.perf_counter()
    run_steps(e2e_steps)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * B * e2e_steps / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": in_bytes,
           "d2h_bytes_per_step": out_bytes,
           "what": "pinned host frames -> device (copy stream, double-buffered) -> full path -> fields to pinned host"}
    eng.close()

    # ---- single-pair latency (request = host pair in, field out)
    cfg1 = rp.Config.from_schedule(W, H, sched, bit_depth=12, precision=head, max_batch=1)
    eng1 = rp.Engine(cfg1, device=local)
    o1 = eng1.empty_outputs(1)
    h1 = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in o1]
    lat = []
    for k in range(args.latency_requests + 5):
        t0 = time.perf_counter()
        a_in[0][0].copy_(a_host[k % N_DISTINCT], non_blocking=True)
        b_in[0][0].copy_(b_host[k % N_DISTINCT], non_blocking=True)
        eng1.process_pair(a_in[0][0], b_in[0][0], out=o1)
        for o, ho in zip(o1, h1):
            ho.copy_(o, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        if k >= 5:
            lat.append(1000.0 * (time.perf_counter() - t0))
    eng1.close()
    lat.sort()
    latency = {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
               "requests": len(lat), "batch": 1, "what": "pinned host pair -> device -> full path -> field on host"}

    # ---- roofline of the dominant kernel (traced launches of the headline path)
    recs = traces[head]
    passes = [r for r in recs if r["name"].startswith("pass/")]
    dom = max(passes, key=lambda r: r["total_ms"])
    per_launch_ms = dom["total_ms"] / dom["launches"]
    region = ((dom["nx"] - 1) * dom["step"] + dom["window"]) * ((dom["ny"] - 1) * dom["step"] + dom["window"])
    # algorithmic flops: the definition's 2 w^2 (2r+1)^2 per window; the
    # block-decomposed kernel executes 2 (covered pixels) (2r+1)^2 of them
    plane_flops = 2.0 * region * (2 * dom["radius"] + 1) ** 2 * dom["pairs"]
    direct_flops = 2.0 * dom["nx"] * dom["ny"] * dom["window"] ** 2 * (2 * dom["radius"] + 1) ** 2 * dom["pairs"]
    achieved = direct_flops / (per_launch_ms / 1000.0) / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_derived = sms * 128 * 2 * sm_max * 1e6 / 1e12
    fma = measure_fma_peak(local)
    if head == "fp32":
        bound, peak = "alu", fma["tflops"]
        peak_src = (f"measured: FMA microbenchmark {fma['tflops']:.1f} TFLOP/s ({fma['form']} FMAs; scalar "
                    f"{fma['scalar_tflops']:.1f}, packed f32x2 {fma['packed_tflops']:.1f}) at "
                    f"{(fma['clocks'] or {}).get('sm_mhz')} MHz (derived {sms} SMs x 128 lanes x 2 x "
                    f"{sm_max:.0f} MHz = {fp32_derived:.1f})")
    else:
        bound = "tensor"
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        peak_src = "measured (MEASURED_PEAKS.json bf16_tflops_sustained)" if peaks else "fallback"
    traffic = stored_traffic(args.workload, head, dom)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"pass_kernel {dom['name']} (w={dom['window']}, s={dom['step']}, "
                f"r={dom['radius']}, {dom['pairs']} pairs/launch)", "peak_source": peak_src,
                "per_launch_ms": per_launch_ms, "algorithmic_flops_per_launch": direct_flops,
                "executed_flops_per_launch": plane_flops,
                "executed_frac": plane_flops / (per_launch_ms / 1000.0) / 1e12 / peak,
                "fp32_fma_peak": fma, "fp32_derived_peak_tflops": fp32_derived}
    stage_ms = {r["name"]: r["total_ms"] / r["launches"] for r in recs}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    kernels = kernel_roofline(recs, 2, 8, hbm_peak)  # u16 frames, margin 8 (radius 4)
    launches_per_step = sum(r["launches"] for r in recs) / 3.0

    # ---- CPU baseline and accuracy against the FP64 oracle
    cpu = None
    accuracy = {}
    if pool is not None:
        sample_seeds = [1002 + k for k in range(cores)]
        dt, res = oracle_round(pool, [(sd, args.workload) for sd in sample_seeds])
        pool.close()
        cpu = {"value": len(sample_seeds) / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(sample_seeds)} pairs of the workload, one per core, FP64 oracle, "
                         f"{dt:.1f} s wall"}
        ref = {r[0]: r for r in res}
        if seeds[0] in ref:
            ru, rv = ref[seeds[0]][2], ref[seeds[0]][3]
            for prec, (u, v) in fields.items():
                err = np.maximum(np.abs(u - ru), np.abs(v - rv))
                accuracy[prec] = {"p99_px": float(np.percentile(err, 99)), "max_px": float(err.max()),
                                  "within_1e-3": float(np.mean(err <= 1e-3)),
                                  "over_0.01": float(np.mean(err > 1e-2))}
    for prec in paths:
        if prec in accuracy:
            paths[prec]["err_vs_oracle"] = accuracy[prec]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": paths[head]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": head, "data": "synthetic",
            "config": {"workload": workload, "batch_pairs_per_gpu": B, "precision": head,
                       "l2": f"inputs {in_bytes / 2**20:.0f} MiB per step > 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "paths": paths, "latency": latency, "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clocks, "gpu_launches": int(round(launches_per_step * args.steps)),
            "stage_ms_per_launch": stage_ms,
            "kernel_roofline": {"peak_gbs": hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs", "rows": kernels},
            "vectors_per_s": value * 127 * 127,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def kernel_bytes(rec: dict, bpp: int, margin: int) -> int | None:
    """Algorithmic DRAM bytes of one traced launch (the data the step must
    move, independent of how the kernel schedules it): frames read once and
    written once, node fields read and written once.  rec: a stage-trace record
    (name, pairs, image size, grid)."""
    name, n, W, H = rec["name"], rec["pairs"], rec["width"], rec["height"]
    nodes = rec["nx"] * rec["ny"]
    if name == "ingest":  # u8/u16 frame in, float frame (interior) out
        return n * W * H * (bpp + 4)
    if name.startswith("down/"):  # a frame in (the input format at level 1, float above), its half out
        src = bpp if name == "down/L1" else 4
        return n * (W * H * src + (W // 2) * (H // 2) * 4)
    if name.startswith("deform"):  # frame in, warped float frame with margins out
        src = 4 if "/L" in name else bpp
        return n * (W * H * src + (W + 2 * margin) * (H + 2 * margin) * 4)
    if name.startswith("uod/"):  # u, v, info in; u, v, mask out
        return n * nodes * 21
    if name.startswith("interp/"):  # u, v out (and the coarser field in)
        return n * nodes * 16
    if name == "vort":  # u, v in; vorticity out
        return n * nodes * 12
    if name.startswith("pass/"):  # frames A and B' read (the pass is bound by the ALU)
        return n * W * H * 4 * 2
    return None


def kernel_roofline(recs: list, bpp: int, margin: int, hbm_gbs: float) -> list:
    """Achieved bandwidth of every traced kernel against the measured HBM peak."""
    rows = []
    for r in recs:
        b = kernel_bytes(r, bpp, margin)
        ms = r["total_ms"] / r["launches"]
        if b is None or ms <= 0:
            continue
        gbs = b / (ms * 1e-3) / 1e9
        rows.append({"kernel": r["name"], "ms_per_launch": round(ms, 4), "bytes_per_launch": b,
                     "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_gbs, 3),
                     "bound": "alu" if r["name"].startswith("pass/") else "hbm"})
    return rows


def stored_traffic(workload: str, head: str, dom: dict, path: str | None = None):
    """DRAM bytes per launch of the dominant pass from ncu counters stored in
    profiles/traffic.json, or None.  An entry counts only for the workload,
    precision and pass it was taken on, with the same window, step and radius,
    and while the pass kernels' code is the code it was taken on."""
    try:
        with open(path or os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh)
        ent = tr.get(f"{workload}/{head}/{dom['name']}")
        if (ent and ent.get("source_hash") == _kernel_source_hash()
                and (ent.get("window"), ent.get("step"), ent.get("radius")) ==
                (dom["window"], dom["step"], dom["radius"])):
            return ent["bytes_per_pair"] * dom["pairs"]
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return None


def _kernel_source_hash() -> str:
    """Hash of the pass kernels' code with comments and whitespace removed, so
    that stored DRAM counters stay tied to the code they were taken on and
    survive edits to comments alone."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("pass_impl.cuh", "tc_pass.cuh", "k_pass_fp32.cu", "k_pass_tc.cu", "pass_plan.cpp"):
        with open(os.path.join(ROOT, "paper_2504_17987_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip())
        h.update(text.encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
