#!/usr/bin/env python
"""Throughput of the deep-octree ray caster on GB300: Mrays/s and stereo frames/s.

Workload (default): the depth-24 canvas of 40 km (finest cell 2.4 mm) built
from 210,000 seeded sphere stamps, rendered as a stereo pair of 2160 x 2160
per eye from inside a 1 m room (synth config 2). One step = one render of
both eyes through the C ABI (one persistent launch of the mixed-precision
kernel). The canvas is resident in HBM before timing; L2 is flushed (256 MB
write) before every timed step, and each step is timed with CUDA events on
the launching stream.

Also reported: the plain FP64 GPU path (one launch per view) on the same
views, the max abs error against the FP64 oracle on a seeded pixel sample,
the end-to-end rate through canvox_render_host (view table up, image down),
the roofline of the traversal kernel and the oracle timed on the host cores.

  python bench.py [--gpus N --steps K --warmup W --impl {canvox,reference} --config C]
Under torchrun each rank renders its own copy of the workload (replicas:
weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s and stereo frames/s at depth 24-27 vs plain FP64 GPU path; max err vs FP64"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["canvox", "reference"], default="canvox")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline sample")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 baseline, e2e and CPU baseline")
    ap.add_argument("--no-deep", action="store_true", help="skip the depth-27 workloads (configs 3 and 4)")
    ap.add_argument("--opts", type=str, default="", help="render options as JSON")
    ap.add_argument("--no-autotune", action="store_true", help="time the built-in default schedule")
    ap.add_argument("--res-scale", type=float, default=1.0, help="shrink every image side (profiling cases)")
    ap.add_argument("--n-fine", type=int, default=0, help="fine stamps of configs 2-4 (profiling cases; 0 = config)")
    ap.add_argument("--paint-only", action="store_true",
                    help="time the device stamp painter on the config's stamp table and exit")
    ap.add_argument("--oracle-full", action="store_true",
                    help="with --impl reference: time the oracle once over the whole frame (all host cores)")
    return ap.parse_args()


def workload_name(cid):
    import synth
    return synth.CONFIGS[cid]["name"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def profiled_counters(cid, res_scale, n_fine):
    """Per-launch hardware counters of the traversal kernel from the committed ncu summary (DRAM bytes, L2
    bytes, warp and thread instructions), or None when the summary is for another workload or the kernel
    source has changed since it was captured."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "mixed_kernel_c2_counters.txt")
    if cid != 2 or res_scale != 1.0 or n_fine or not os.path.exists(p):
        return None
    src = os.path.join(ROOT, "paper_1704_02724_gb300", "csrc", "trace_mixed.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    fields = {}
    with open(p) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("kernel_sha256") != sha:
        return None
    ctr = {k: float(fields[k]) for k in ("dram_bytes_per_launch", "lts_bytes_per_launch", "warp_inst_per_launch",
                                         "thread_inst_per_launch", "steps_per_launch")}
    ctr["stalls"] = {k[len("stall_share_"):]: float(v) for k, v in fields.items() if k.startswith("stall_share_")}
    return ctr


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def oracle_rate(canvas, cams, budget_s, seed=12345, threads=0):
    """Time the FP64 oracle on a seeded pixel sample sized for ~budget_s (threads 0: all host cores)."""
    import oracle
    import synth
    threads = threads or oracle.max_threads()
    total = synth.total_pixels(cams)
    rng = np.random.default_rng(seed)
    order = rng.permutation(total).astype(np.int64)
    n, spent, done, out = 256, 0.0, 0, []
    t_start = time.perf_counter()
    while done < total:
        px = order[done:done + n]
        t = time.perf_counter()
        out.append((px, oracle.render(canvas, cams, px_idx=px, threads=threads, counters=True)))
        dt = time.perf_counter() - t
        spent += dt
        done += len(px)
        if spent >= budget_s:
            break
        rate = len(px) / max(dt, 1e-9)
        n = int(min(max(256, rate * (budget_s - spent) * 0.5), 1 << 20))
    wall = time.perf_counter() - t_start
    px = np.concatenate([p for p, _ in out])
    ref = np.concatenate([r[0] for _, r in out])
    counts = {"steps": np.concatenate([r[1][:, 0] for _, r in out]),
              "length": np.concatenate([r[2][:, 1] for _, r in out])}
    return px, ref, done / wall / 1e6, wall, threads, counts


def binned(values, keys, edges):
    """Median and max of values per [edges[i], edges[i+1]) bin of keys (empty bins left out)."""
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (keys >= lo) & (keys < hi)
        if np.any(m):
            v = values[m]
            rows.append({"from": lo, "to": hi, "n": int(m.sum()), "median": float(np.median(v)),
                         "max": float(v.max())})
    return rows


def aggregate_ranks(ms_step, rays, world, device=None):
    """Whole-job throughput: the slowest rank's time per step, all ranks' rays (replicas, weak scaling).
    Returns (max ms per step over ranks, Mrays/s of the job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_step), float(rays)], dtype=torch.float64, device=device)
    if world > 1:
        m = t[0:1].clone()
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        n = t[1:2].clone()
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        t = torch.cat([m, n])
    ms_max, total_rays = float(t[0].item()), float(t[1].item())
    return ms_max, total_rays / (ms_max * 1e-3) / 1e6


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    cid = args.config
    canvas = synth.build_config(cid)
    cams = synth.config_cameras(cid)
    import oracle
    total = synth.total_pixels(cams)
    if args.oracle_full:
        t = time.perf_counter()
        oracle.render(canvas, cams, threads=oracle.max_threads())
        sec = time.perf_counter() - t
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": total / sec / 1e6, "unit": "Mrays/s",
                          "config": {"workload": workload_name(cid), "rays_per_frame": total},
                          "cpu_baseline": {"value": total / sec / 1e6, "unit": "Mrays/s", "cores": oracle.max_threads(),
                                           "kind": "oracle", "sample": "the whole frame, once"},
                          "seconds": sec}), flush=True)
        return 0
    rng = np.random.default_rng(777)
    # each step: a bounded sample of the workload, sized so that warmup + steps end within minutes
    probe = rng.choice(total, size=512, replace=False).astype(np.int64)
    t = time.perf_counter()
    oracle.render(canvas, cams, px_idx=probe)
    rate = 512 / max(time.perf_counter() - t, 1e-6)
    per_step = int(max(256, min(total, rate * 120.0 / max(1, args.steps + args.warmup))))
    times = []
    for k in range(args.warmup + args.steps):
        px = rng.choice(total, size=per_step, replace=False).astype(np.int64)
        t = time.perf_counter()
        oracle.render(canvas, cams, px_idx=px)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    sec = sum(times) / len(times)
    value = per_step / sec / 1e6
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp64", "data": "synthetic",
        "config": {"workload": workload_name(cid), "rays_per_frame": total, "step_sample_rays": per_step},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} seeded random pixels of the {total}-ray frame per step"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


BUILTIN_SCHEDULE = {"tile_w": 8, "frame_levels": 20, "refill": 0, "block_threads": 256, "blocks_per_sm": 0,
                    "smem_records": 0, "traversal": 0}


def deep_oracle(samples):
    """Spawned helper of deep_workloads (host cores only): the host painter's pools of the depth-27 canvas and the
    oracle on the sampled pixels of configs 3 and 4. Returns ({config: rgba [n, 4]}, host painter seconds)."""
    import oracle
    import synth
    t = time.perf_counter()
    canvas = synth.build_config(3)
    host_s = time.perf_counter() - t
    return {cid: oracle.render(canvas, synth.config_cameras(cid), px_idx=px) for cid, px in samples.items()}, host_s


def deep_workloads(cx, synth, torch, stream, flush, dev, topts, steps=5):
    """The depth-27 canvas of 1,000,000 fine stamps (configs 3 and 4), painted on the GPU from its stamp table;
    config 3's eight stereo pairs in one persistent launch replayed from a CUDA graph, config 4's 64 uneven views
    batched (one launch), one launch per view, with the built-in schedule and with the schedule the autotuner picks
    for them. Max error against the oracle on seeded pixel samples; the oracle reads the host painter's pools of the
    same stamps, built and rendered in a spawned process while the GPU is timed."""
    import concurrent.futures
    import multiprocessing
    out = {}
    cams = {cid: synth.config_cameras(cid) for cid in (3, 4)}
    samples = {}
    for cid in (3, 4):
        n_px = synth.total_pixels(cams[cid])
        rng = np.random.default_rng(1704 + cid)
        samples[cid] = np.sort(rng.choice(n_px, size=min(n_px, 200000), replace=False)).astype(np.int64)
    pool = concurrent.futures.ProcessPoolExecutor(max_workers=1, mp_context=multiprocessing.get_context("spawn"))
    fut = pool.submit(deep_oracle, samples)
    D, E, c, r, q, _ = synth.config_stamps(3)
    t = time.perf_counter()
    nr, nl = cx.paint_spheres(D, E, c, r, q)
    paint_s = time.perf_counter() - t

    def timed(cid, o):
        img = torch.empty((synth.total_pixels(cams[cid]), 4), dtype=torch.float32, device=dev)
        for _ in range(3):
            cx.render(cams[cid], img, **o)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cx.render(cams[cid], img, **o)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = statistics.median(ms)
        sampled = img[torch.from_numpy(samples[cid]).to(dev)].cpu().numpy().astype(np.float64)
        return {"Mrays_s": img.shape[0] / (m * 1e-3) / 1e6, "ms": m}, sampled

    res3, img3 = timed(3, dict(topts, use_graph=1))
    res4 = {}
    res4["batched"], img4 = timed(4, dict(topts))
    res4["per_view"], _ = timed(4, dict(topts, per_view=1))
    res4["builtin_schedule"], _ = timed(4, dict(topts, **BUILTIN_SCHEDULE))
    t = time.perf_counter()
    best = cx.autotune(cams[4])
    tune_s = time.perf_counter() - t
    tuned = {k: best[k] for k in BUILTIN_SCHEDULE}
    res4["autotuned_on_c4"], _ = timed(4, dict(topts, **tuned))
    refs, host_s = fut.result()
    pool.shutdown()
    for cid, res, img in ((3, {"graph": res3}, img3), (4, res4, img4)):
        err = np.abs(img - refs[cid]).max(axis=1)
        key = f"c{cid}"
        out[key] = {"workload": synth.CONFIGS[cid]["name"] + f" ({len(cams[cid])} views, {synth.total_pixels(cams[cid])}"
                                                               f" rays, depth {D}, {nr} records, {nl} leaves)",
                    "timings": res, "max_err_vs_oracle": float(err.max()), "pixels_over_1e-5": int(np.sum(err > 1e-5)),
                    "oracle_pixels": int(samples[cid].size), "l2": "flushed before every timed render",
                    "schedule": "the one autotuned on c2 unless the timing's name says otherwise"}
    out["c3"]["stereo_fps"] = 8 / (res3["ms"] * 1e-3)
    out["c3"]["device_painter_seconds"] = round(paint_s, 2)
    out["c3"]["host_painter_seconds"] = round(host_s, 1)
    out["c4"]["batched_over_per_view"] = res4["per_view"]["ms"] / res4["batched"]["ms"]
    out["c4"]["autotuned_over_builtin"] = res4["builtin_schedule"]["ms"] / res4["autotuned_on_c4"]["ms"]
    out["c4"]["autotune"] = dict(tuned, seconds=round(tune_s, 1))
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_1704_02724_gb300 as cx
    import synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    cid = args.config
    if args.paint_only:
        D_, E_, c_, r_, q_, _ = synth.config_stamps(cid, n_fine=args.n_fine or None)
        cx.paint_spheres(D_, E_, c_[:8], r_[:8], q_[:8])   # warm-up (module load, allocator)
        torch.cuda.synchronize()
        t_dev = time.perf_counter()
        nr_, nl_ = cx.paint_spheres(D_, E_, c_, r_, q_)
        print(json.dumps({"metric": "device stamp painter", "value": time.perf_counter() - t_dev, "unit": "s",
                          "higher_is_better": False, "config": {"workload": workload_name(cid),
                                                                "stamps": int(r_.shape[0])},
                          "records": nr_, "leaves": nl_}), flush=True)
        return 0
    opts = json.loads(args.opts) if args.opts else {}
    t_host = time.perf_counter()
    canvas = synth.build_config(cid, n_fine=args.n_fine or None)
    host_paint_s = time.perf_counter() - t_host
    cams = synth.config_cameras(cid, res_scale=args.res_scale)
    n_px = synth.total_pixels(cams)
    cx.upload_octree(canvas.nodes, canvas.leaves, canvas.depth, canvas.extent)
    h_hash, d_hash = cx.octree_hash()
    out = torch.empty((n_px, 4), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_autotune and not opts:
        # the schedule (tile shape, refill, shared-memory prefix, frame depth, traversal) picked by
        # the library's autotuner on these views; it becomes the default for the renders below
        t_tune = time.perf_counter()
        tuned = cx.autotune(cams)
        tuned["seconds"] = round(time.perf_counter() - t_tune, 1)
    # timed renders skip the per-lane read counters (instrumentation, not work); one counted render of the
    # same views after the timed region gives the algorithmic bytes (the traversal is deterministic)
    topts = dict({"count_reads": 0}, **opts)
    for _ in range(max(3, args.warmup)):
        cx.render(cams, out, **topts)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        cx.render(cams, out, **topts)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = sum(ms) / len(ms)
    cx.render(cams, out, **dict(topts, count_reads=1))
    torch.cuda.synchronize()
    stats = cx.get_stats(check=False)
    rays = stats["rays"]
    ms_max, value = aggregate_ranks(ms_step, rays, world, dev)

    line = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        algo_bytes = 32 * stats["slot_reads"] + 8 * stats["leaf_loads"] + 16 * stats["rays"]
        achieved = algo_bytes / (ms_step * 1e-3) / 1e9
        ctr = profiled_counters(cid, args.res_scale, args.n_fine)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        clk_mhz = (clk or {}).get("sm_mhz") or 2070.0
        issue_peak = n_sm * 4 * clk_mhz * 1e6 / 1e9   # warp instructions per second, G: one per scheduler per cycle
        roofline = {
            # the bytes roof of the formula: algorithmic bytes per launch over the measured HBM copy bandwidth
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ctr["dram_bytes_per_launch"] if ctr else None, "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": algo_bytes, "bytes_formula": "32*slot_reads + 8*leaf_loads + 16*rays",
            "bound_note": "what binds is instruction issue (ncu: 0.84 of the issue peak on this launch, ALU the busiest pipe, "
                          "DRAM ~0.2 % of the algorithmic bytes): see 'issue'; the gathers are served by L1/L2",
        }
        if ctr:
            # counters of this launch from the committed ncu capture (same kernel source, same schedule)
            roofline["issue"] = {
                "achieved": ctr["warp_inst_per_launch"] / (ms_step * 1e-3) / 1e9, "peak": issue_peak,
                "unit": "G warp-instructions/s", "frac": ctr["warp_inst_per_launch"] / (ms_step * 1e-3) / 1e9 / issue_peak,
                "peak_kind": f"derived: {n_sm} SMs x 4 schedulers x 1 warp-instruction/cycle x {clk_mhz:.0f} MHz (sampled)",
                "thread_inst_per_leaf_step": ctr["thread_inst_per_launch"] / ctr["steps_per_launch"],
                "warp_inst_per_leaf_step": ctr["warp_inst_per_launch"] / ctr["steps_per_launch"]}
            roofline["l2"] = {"achieved": ctr["lts_bytes_per_launch"] / (ms_step * 1e-3) / 1e9, "unit": "GB/s",
                              "note": "lts__t_bytes per launch (ncu) over the timed launch; see l2_gather for the probe"}
            if ctr["stalls"]:
                roofline["stalls"] = {
                    "memory_latency": ctr["stalls"].get("long_scoreboard"), "share_of_stall_cycles": ctr["stalls"],
                    "note": "ncu stall reasons of the same kernel source on the reduced stereo case (--set full); "
                            "memory_latency = long scoreboard (L1/L2 gathers, spilled words)"}
        line = {
            "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32+fp64", "data": "synthetic",
            "config": {"workload": workload_name(cid) + (f" [reduced: res x{args.res_scale}, n_fine {args.n_fine}]"
                                                         if args.res_scale != 1.0 or args.n_fine else "")
                       + f" ({len(cams)} views, {n_px} rays, depth {canvas.depth},"
                       f" {canvas.n_records} records, {canvas.n_leaves} leaves)",
                       "rays_per_step": rays * world, "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": f"replicas x{world}", "opts": cx.default_opts() | topts,
                       "schedule": "autotuned" if tuned else ("given" if opts else "built-in default")},
            "stereo_fps": (world / (ms_max * 1e-3)) if len(cams) == 2 else None,
            "wall_ms_per_step_incl_flush": wall * 1e3 / args.steps,
            # per render: the eye-path kernel and the traversal kernel (one per view in per-view mode)
            "gpu_launches": args.steps * (1 + (1 if not opts.get("per_view") else len(cams))),
            "roofline": roofline,
            "stats": {k: v for k, v in stats.items() if k != "status"},
            "hash_ok": h_hash == d_hash,
            "autotune": tuned,
            "clocks": clk,
        }
    if rank == 0 and not args.no_extras and world == 1:
        # plain FP64 GPU path on the same views (one launch per view)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out64 = torch.empty_like(out)
        cx.render(cams, out64, precision=cx.PREC_FP64)
        torch.cuda.synchronize()
        f64 = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            cx.render(cams, out64, precision=cx.PREC_FP64)
            e1.record(stream)
            torch.cuda.synchronize()
            f64.append(e0.elapsed_time(e1))
        ms64 = statistics.median(f64)
        line["fp64_plain"] = {"value": rays / (ms64 * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms64,
                              "speedup_of_mixed": ms64 / ms_step}
        # the FP64 twin of the mixed traversal (same links, queue and schedule; FP64 arithmetic): what the
        # precision scheme alone buys
        out64l = torch.empty_like(out)
        cx.render(cams, out64l, precision=cx.PREC_FP64_LINKS, count_reads=0)
        torch.cuda.synchronize()
        f64l = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            cx.render(cams, out64l, precision=cx.PREC_FP64_LINKS, count_reads=0)
            e1.record(stream)
            torch.cuda.synchronize()
            f64l.append(e0.elapsed_time(e1))
        ms64l = statistics.median(f64l)
        line["fp64_links"] = {"value": rays / (ms64l * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms64l,
                              "speedup_of_mixed": ms64l / ms_step}
        out32 = torch.empty_like(out)
        cx.render(cams, out32, precision=cx.PREC_FP32)
        torch.cuda.synchronize()
        # end to end through canvox_render_host: view table up, image down, every step
        host = torch.empty((n_px, 4), dtype=torch.float32, pin_memory=True)
        cx.render_host(cams, host, **topts)
        k_e2e = min(args.steps, 10)
        t = time.perf_counter()
        for _ in range(k_e2e):
            cx.render_host(cams, host, **topts)
        e2e_s = (time.perf_counter() - t) / k_e2e
        st2 = cx.get_stats(check=False)
        line["e2e"] = {"value": rays / e2e_s / 1e6, "unit": "Mrays/s", "h2d_bytes_per_step": st2["h2d_bytes"],
                       "d2h_bytes_per_step": st2["d2h_bytes"], "ms_per_step": e2e_s * 1e3}
        # the paper's FP32 walks (Sec. 6.3): cell-local and canvas-coordinate, with ray-angle errors
        walks = {}
        for name, prec in (("cell32", cx.PREC_CELL32), ("world32", cx.PREC_WORLD32), ("cell16", cx.PREC_CELL16)):
            img_w = torch.empty_like(out)
            ang = torch.zeros(n_px, dtype=torch.float32, device=dev)
            e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0_.record(stream)
            cx.render(cams, img_w, precision=prec, angle_deg=ang)
            e1_.record(stream)
            torch.cuda.synchronize()
            a = ang.cpu().numpy().astype(np.float64)
            walks[name] = {"image": img_w, "ms": e0_.elapsed_time(e1_), "angles": a,
                           "angle_deg_max": float(a.max()), "angle_deg_p99_9": float(np.percentile(a, 99.9)),
                           "angle_deg_median": float(np.median(a))}
        # measurement helpers: L2 sector-gather and FP64 probes, the frame's footprint (compulsory bytes)
        l2_gbs = cx.probe_l2_gather()
        line["l2_gather"] = {"probe_gbs": l2_gbs, "achieved_gbs": achieved, "frac": achieved / l2_gbs,
                             "note": "algorithmic bytes against random 32 B sector gathers from a half-L2 buffer,"
                                     " L1 bypassed"}
        if "l2" in line["roofline"]:
            line["roofline"]["l2"]["probe_gbs"] = l2_gbs
            line["roofline"]["l2"]["frac"] = line["roofline"]["l2"]["achieved"] / l2_gbs
        line["fp64_probe_gflops"] = cx.probe_fp64()
        t_fp = time.perf_counter()
        n_rec_fp, n_leaf_fp = cx.footprint(cams)
        line["footprint"] = {"records": n_rec_fp, "leaves": n_leaf_fp,
                             "compulsory_bytes": 32 * n_rec_fp + 8 * n_leaf_fp,
                             "with_links_bytes": 80 * n_rec_fp + 8 * n_leaf_fp,
                             "dram_bytes_per_launch": line["roofline"]["traffic"],
                             "seconds": round(time.perf_counter() - t_fp, 1)}
        # FP64 oracle on host cores: CPU baseline and the error of each GPU path on its sample
        px, ref, rate, wall_s, cores, counts = oracle_rate(canvas, cams, args.cpu_seconds)
        img = out.cpu().numpy().astype(np.float64)[px]
        err = np.abs(img - ref).max(axis=1)
        line["cpu_baseline"] = {"value": rate, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                                "sample": f"{len(px)} seeded random pixels of the {n_px}-ray frame, {wall_s:.1f} s"}
        line["max_err_vs_oracle"] = {
            "mixed": float(err.max()), "mixed_pixels_over_1e-5": int(np.sum(err > 1e-5)),
            "fp64_plain": float(np.abs(out64.cpu().numpy().astype(np.float64)[px] - ref).max()),
            "fp64_links": float(np.abs(out64l.cpu().numpy().astype(np.float64)[px] - ref).max()),
            "fp32_plain": float(np.abs(out32.cpu().numpy().astype(np.float64)[px] - ref).max()),
            "pixels": int(len(px))}
        for name, w in walks.items():
            w["max_err_vs_oracle"] = float(np.abs(w.pop("image").cpu().numpy().astype(np.float64)[px] - ref).max())
            w["Mrays_s"] = rays / (w.pop("ms") * 1e-3) / 1e6
            # ray-angle error against the ray's length in the canvas and the cells it crossed (oracle sample)
            a = w.pop("angles")[px]
            w["angle_vs_length_m"] = binned(a, counts["length"], [1e-3, 1e-2, 1e-1, 1, 10, 100, 1e3, 1e4, 1e5])
            w["angle_vs_cells"] = binned(a, counts["steps"], [1, 10, 100, 1000, 10000, 100000])
        line["paper_fp32_walks"] = walks
        # the oracle on one core (a smaller sample; the all-core figure above is the baseline)
        _, _, rate1, wall1, _, _ = oracle_rate(canvas, cams, max(2.0, args.cpu_seconds / 3), seed=54321, threads=1)
        line["cpu_baseline_1core"] = {"value": rate1, "unit": "Mrays/s", "cores": 1, "seconds": round(wall1, 1)}
        # the device stamp painter on the same stamp table (replaces the uploaded canvas; last)
        D_, E_, c_, r_, q_, _ = synth.config_stamps(cid, n_fine=args.n_fine or None)
        cx.paint_spheres(D_, E_, c_[:8], r_[:8], q_[:8])   # warm-up (module load, allocator)
        torch.cuda.synchronize()
        t_dev = time.perf_counter()
        nr_, nl_ = cx.paint_spheres(D_, E_, c_, r_, q_)
        dev_paint_s = time.perf_counter() - t_dev
        nodes_, leaves_ = cx.download_octree()
        same_full = bool(np.array_equal(nodes_, canvas.nodes) and np.array_equal(leaves_, canvas.leaves))
        # the editing path: the last 1,000 stamps appended to a canvas painted from the others
        k_ = max(0, r_.shape[0] - 1000)
        cx.paint_spheres(D_, E_, c_[:k_], r_[:k_], q_[:k_])
        t_app = time.perf_counter()
        cx.paint_append(c_[k_:], r_[k_:], q_[k_:])
        app_s = time.perf_counter() - t_app
        nodes_, leaves_ = cx.download_octree()
        same_app = bool(np.array_equal(nodes_, canvas.nodes) and np.array_equal(leaves_, canvas.leaves))
        line["device_painter"] = {
            "stamps": int(r_.shape[0]), "seconds": round(dev_paint_s, 3), "records": nr_, "leaves": nl_,
            "host_painter_seconds": round(host_paint_s, 2), "host_threads": os.cpu_count(),
            "identical_to_host_pools": same_full and same_app,
            "append_last_stamps": int(r_.shape[0] - k_), "append_seconds": round(app_s, 3),
            "append_h2d_bytes": int((r_.shape[0] - k_) * 56)}
        if cid == 2 and not args.no_deep:
            del canvas
            line.update(deep_workloads(cx, synth, torch, stream, flush, dev, topts))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
