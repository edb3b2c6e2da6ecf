#!/usr/bin/env python3
"""Benchmark of one IR + reverb-parameter update; the default is the large workload.

Large (default): procedural city of 64 x 64 buildings plus a ground grid (2,015,232
triangles), 8 bands, 256 sources, 1 listener; 1,000,000 primary rays x 200
reflections with the unused segment budget refilled (Section 5: every update traces
the same N x M segments; open scenes end most paths early), IR 3 s at 1 kHz (3000
bins), SH order 3 (16 coefficients).  --workload medium: the furnished hall (24,012
triangles, 16 sources, 200k x 64, IR 2 s, SH order 2, no refill).  --workload paper:
the paper's operating point on a city-like scene.  One step is one whole update
through the C ABI: trace (paths, diffuse-rain shadow rays, histogram accumulation,
direct sound) + estimate (reverb parameters of every source and band), with a new
Philox key per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.  Under torchrun each rank
runs its own independent updates on its GPU (no collective in the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray segments/s; IR+reverb-param updates/s at ≤5% decay-time err vs plain"
UNIT = "ray segments/s"
LARGE = dict(num_rays=1_000_000, max_order=200, sh_order=3, num_bins=3000, min_order=1, ir_rate_hz=1000.0,
             speed_of_sound=343.0, source_radius=0.5, budget_refill=1)
LARGE_NAME = ("large: procedural city, 64x64 buildings + ground (2,015,232 tris), 8 bands, 256 sources, "
              "1M rays x 200 reflections with budget refill, IR 3 s @ 1 kHz, SH order 3")
MEDIUM = dict(num_rays=200_000, max_order=64, sh_order=2, num_bins=2000, min_order=1, ir_rate_hz=1000.0,
              speed_of_sound=343.0, source_radius=0.5)
MEDIUM_NAME = ("medium: furnished hall 40x30x12 m + 2000 boxes (24,012 tris), 8 bands, 16 sources, "
               "200k rays x 64 reflections, IR 2 s @ 1 kHz, SH order 2")
# the paper's operating point (Sec. 5 and 6): 50 primaries x 200 reflections with the unused
# segment budget refilled (10,000 segments per frame), 4 bands, IR at 100 Hz, SH order 1,
# reflections below order 3 left to the early-reflection path; city-like scene, 13 sources
PAPER = dict(num_rays=50, max_order=200, sh_order=1, num_bins=300, min_order=3, ir_rate_hz=100.0,
             speed_of_sound=343.0, source_radius=0.5, budget_refill=1)
PAPER_NAME = ("paper operating point: procedural city, 64x64 buildings + ground (1,032,192 tris), 4 bands, "
              "13 sources, 50 rays x 200 reflections with budget refill, IR 3 s @ 100 Hz, SH order 1, min order 3")
WORKLOADS = {"large": (LARGE, LARGE_NAME, "city"), "medium": (MEDIUM, MEDIUM_NAME, "furnished_hall"),
             "paper": (PAPER, PAPER_NAME, "paper_city")}
WORKLOAD, WORKLOAD_NAME, SCENE = dict(LARGE), LARGE_NAME, "city"
# Algorithmic work of BVH traversal, counted on the pipe that bounds it.  A node visit
# slab-tests two child boxes.  With the ray's direction signs known, each axis has a
# near and a far plane: per box the entry is the largest of the three near-plane
# distances and t_min, the exit the smallest of the three far-plane distances and t_max
# (two three-input max and two three-input min instructions) and entry <= exit is
# checked: 5 FP32 min/max/compare instructions per box, 10 per visit.  A triangle test
# decides with 7 compares (det != 0, u, v, u + v, t_min < t < t_max).  These issue on
# the ALU pipe; the 6 plane distances per box (12 FMA per visit) and the triangle
# arithmetic (about 36 FMA-pipe instructions) go to the FMA pipe, reported beside.
ALU_OPS_PER_NODE = 10.0
ALU_OPS_PER_TRI = 7.0
FMA_OPS_PER_NODE = 12.0
FMA_OPS_PER_TRI = 36.0
# DRAM bytes (read + write) of the shadow-ray launches (k_shadow_packet, the default
# mode) of one update in an ncu capture at fewer primaries, and the shadow rays those
# launches traced; a full-size update is credited with the same bytes per shadow ray.
NCU_SHADOW_DRAM = {"medium": (96_559_360 + 20_052_736, 18_874_205),
                   "large": (248_466_944 + 106_848_256, 478_253_471)}
# warp instructions (smsp__inst_executed.sum) of the same captures, and their shadow rays
NCU_SHADOW_INST = {"medium": (1_518_944_434, 18_874_205), "large": (26_590_588_617, 478_253_471)}


def issue_roofline(workload: str, kernel: str, shadow_rays: float, seconds: float, sms: int, sm_mhz):
    """The shadow-ray kernel against the SMs' instruction issue: warp instructions per shadow
    ray from the ncu capture at fewer primaries, times the update's shadow rays, over the
    kernel's time; the peak is one warp instruction per clock on each of an SM's four
    schedulers.  None when there is no capture for the workload or no clock."""
    ins = NCU_SHADOW_INST.get(workload)
    if kernel != "shadow" or not ins or not sm_mhz or seconds <= 0 or sms <= 0:
        return None
    achieved = ins[0] / ins[1] * shadow_rays / seconds / 1e12
    peak = sms * 4 * sm_mhz * 1e6 / 1e12
    return {"achieved": achieved, "peak": peak, "frac": achieved / peak, "unit": "T warp instructions/s",
            "note": "warp instructions per shadow ray from an ncu capture at fewer primaries; peak = SMs x 4 "
                    "schedulers x the median SM clock sampled during the timed steps"}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, f in rows for i in range(4) if f[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(total_ms: float, rank_work: float, device) -> tuple:
    """(max over ranks of the timed milliseconds, sum over ranks of the work units):
    the job's time is its slowest rank's, its work every rank's."""
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=device)
    wsum = torch.tensor([rank_work], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(wsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(wsum[0])


_SCENE_CACHE = {}


def _oracle_scene():
    """The workload's scene and its oracle form, generated once per process."""
    if SCENE not in _SCENE_CACHE:
        import oracle
        from paper_1803_00430_gb300 import scenes
        sc = getattr(scenes, SCENE)()
        _SCENE_CACHE[SCENE] = (sc, oracle.OracleScene.from_scene(sc))
    return _SCENE_CACHE[SCENE]


def cpu_sample(rays: int, threads: int):
    """The oracle on `rays` primaries of the benchmark's workload (with the refill of
    their own segment budget when the workload refills), on `threads` threads.
    Returns (seconds, segments + shadow rays)."""
    import oracle
    sc, osc = _oracle_scene()
    p = oracle.TraceParams(num_rays=rays, max_order=WORKLOAD["max_order"], sh_order=WORKLOAD["sh_order"],
                           num_bins=WORKLOAD["num_bins"], min_order=WORKLOAD["min_order"],
                           ir_rate_hz=WORKLOAD["ir_rate_hz"], seed=0x5EED,
                           budget_refill=WORKLOAD.get("budget_refill", 0))
    t0 = time.perf_counter()
    H, st, _ = oracle.trace_parallel(osc, p, sc.listener, sc.sources, threads=threads)
    dd = oracle.direct(osc, p, sc.listener, sc.sources)
    oracle.estimate(H, dd["energy"], p.ir_rate_hz)
    dt = time.perf_counter() - t0
    return dt, st["segments"] + st["shadow_rays"]


def _sized_sample(threads: int, target_s: float):
    """Primaries for a sample of about target_s seconds on `threads` threads: a probe,
    then up to three rescalings (the probe's fixed costs overstate the time per ray)."""
    # a refilled primary spends its whole budget of max_order segments: probe with fewer
    rays = min(2 if WORKLOAD.get("budget_refill") else 20, WORKLOAD["num_rays"])
    dt, work = cpu_sample(rays, threads)
    for _ in range(4):
        if dt >= 0.5 * target_s or rays >= WORKLOAD["num_rays"]:
            break
        rays = int(min(WORKLOAD["num_rays"], max(rays + 1, rays * target_s / max(dt, 1e-3))))
        dt, work = cpu_sample(rays, threads)
    return rays, dt, work


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _sample_text(rays: int, dt: float) -> str:
    refill = " with the refill of their segment budget" if WORKLOAD.get("budget_refill") else ""
    return (f"{rays} of the {WORKLOAD['num_rays']} primaries of the {WORKLOAD_NAME.split(':')[0]} workload{refill} "
            f"(full scene and sources, {WORKLOAD['max_order']} reflections), trace + estimate, {dt:.1f} s wall")


def cpu_baseline(target_s: float = 12.0, single_s: float = 6.0):
    """The oracle as it stands on all host cores (the CPU throughput baseline) and on
    one thread (the parity reference), each on a bounded sample of the workload."""
    threads = os.cpu_count() or 1
    rays, dt, work = _sized_sample(threads, target_s)
    r1, d1, w1 = _sized_sample(1, single_s)
    return {"value": work / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": _sample_text(rays, dt),
            "cpu_model": cpu_model(), "arch": platform.machine(),
            "single_thread": {"value": w1 / d1, "unit": UNIT, "cores": 1, "sample": _sample_text(r1, d1)}}


def learned_at_bar(ctx) -> dict:
    """The metric's second half: IR + reverberation-parameter updates/s at <= 5 % mean
    decay-time error, for the plain estimator and for the learned one (a network trained
    here, on the method's own IRs), on held-out procedural rooms and corridors whose
    references are the plain estimator at 500k rays; the learned workflow's training
    protocol and ray counts (python -m paper_1803_00430_gb300.learned), so that the two give
    the same numbers; about two minutes.  Near the bar the mean error moves by a few tenths
    of a percent between independent trace sets, which can move a form's crossing by one
    ray count."""
    from paper_1803_00430_gb300 import learned as L
    t0 = time.time()
    rays = [1000, 2000, 4000, 8000, 16000, 32000]  # the workflow's list: the traces' keys follow it
    train = L.make_dataset(ctx, 8192, seed=101, low_rays=[2000, 4000, 8000], high_rays=100000, copies=2)
    test_scenes = L.learned_scenes(202, 512)
    test = L.make_dataset(ctx, 512, seed=202, low_rays=rays, high_rays=500000)
    mlp, _ = L.fit(ctx, train, steps=6000, batch=512, lr=1e-3, weight_decay=1e-2, log_every=6000)
    res = L.sweep(ctx, mlp, test, rays, test_scenes)
    mlp.close()
    out = {"bar": res["bar"], "unit": "updates/s",
           "workload": "512 held-out procedural rooms and corridors, 1 source, 8 bands, 64 reflections, "
                       "SH order 0, IR 2 s at 1 kHz; references: the plain estimator at 500k rays",
           "training": "8192 scenes x (2k, 4k, 8k) rays x 2 copies, labels at 100k rays, 6000 AdamW steps",
           "seconds": round(time.time() - t0, 1)}
    for form, key in (("plain", "plain"), ("learned", "net")):
        n = res[f"rays_at_bar_{key}"]
        e = res["per_rays"][n] if n else {}
        out[form] = {"rays": n, "updates_per_s": res[f"updates_per_s_at_bar_{key}"],
                     "rt_err_mean": e.get(f"rt_err_mean_{key}"), "rt_err_p95": e.get(f"rt_err_p95_{key}")}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    # each step a bounded sample: the whole run stays within about three minutes
    per_step = max(1.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    rays, _, _ = _sized_sample(threads, per_step)
    for _ in range(args.warmup):
        cpu_sample(rays, threads)
    total_t, total_w = 0.0, 0.0
    for _ in range(args.steps):
        dt, w = cpu_sample(rays, threads)
        total_t += dt
        total_w += w
    v = total_w / total_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "sample_rays_per_step": rays},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{rays} primaries of the {WORKLOAD_NAME.split(':')[0]} workload per step"
                                       + (" with the refill of their segment budget"
                                          if WORKLOAD.get("budget_refill") else ""),
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp32-paths", action="store_true", help="time the all-FP32 path precision form")
    ap.add_argument("--shadow-mode", default="auto", choices=["auto", "packets", "lanes"],
                    help="shadow rays as warp packets or one per lane (auto: the library default, packets)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-vs-plain updates/s at the 5 %% decay-time error bar (one GPU only)")
    ap.add_argument("--rays", type=int, default=0, help="primaries per update (default: the workload's; "
                    "smaller values make a small case for profilers)")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS),
                    help="large: the procedural city with budget refill (default); medium: the furnished hall; "
                         "paper: the paper's operating point on a city-like scene")
    args = ap.parse_args()
    global SCENE, WORKLOAD_NAME
    wl, WORKLOAD_NAME, SCENE = WORKLOADS[args.workload]
    WORKLOAD.clear()
    WORKLOAD.update(wl)
    if args.rays:
        WORKLOAD["num_rays"] = args.rays
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_1803_00430_gb300 import build, rpr, scenes
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    rpr.load()
    # oracle timing runs before any further GPU work (a process pool is not used)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    stream = torch.cuda.current_stream()
    ctx = rpr.Context(local, stream)
    sc = getattr(scenes, SCENE)()
    scene = rpr.Scene.from_scene(ctx, sc)
    info = scene.info()
    S, B = sc.num_sources, sc.num_bands
    flags = rpr.RP_FLAG_DEVICE_POSITIONS | (rpr.RP_FLAG_FP32_PATHS if args.fp32_paths else 0)
    flags |= {"auto": 0, "packets": rpr.RP_FLAG_SHADOW_PACKETS, "lanes": rpr.RP_FLAG_SHADOW_LANES}[args.shadow_mode]
    base = rpr.TraceParams(**WORKLOAD, flags=flags, scene_id=rank)
    K, T = base.K, base.num_bins
    out = rpr.DeviceTrace(S, B, K, T)
    params = torch.empty(S * B * C_sizeof("rp_reverb_params"), dtype=torch.uint8, device="cuda")
    lis_d = torch.tensor(sc.listener, device="cuda")
    src_d = torch.tensor(sc.sources, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    rpr.check(ctx.lib.rp_trace_reserve(scene.h, ctypes.byref(base.c()), S), "reserve")
    # measured FP32 pipe throughput (calibration for the roofline; untimed)
    fma_peak, minmax_peak = ctx.pipe_peaks()

    def step(i):
        p = base.c()
        p.seed = scenes.PHILOX_KEY_BASE + i
        rpr.check(ctx.lib.rp_trace(scene.h, ctypes.byref(p), rpr._ptr(lis_d), rpr._ptr(src_d), S,
                                   rpr._ptr(out.H), rpr._ptr(out.direct), rpr._ptr(out.stats), None), "rp_trace")
        ep = rpr.rp_estimate_params(base.ir_rate_hz, 0.1, 3.0)
        rpr.check(ctx.lib.rp_estimate(ctx.h, rpr._ptr(out.H), rpr._ptr(out.direct), S, B, K, T,
                                      ctypes.byref(ep), rpr._ptr(params), None), "rp_estimate")

    for i in range(args.warmup):
        step(i)
    rpr.check(ctx.sync_status(), "warmup")

    # per-kernel events (library side, on the same stream) during the timed region
    ctx.profile(True)
    ctx.profile_reset()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    work_steps = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(args.warmup + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    rpr.check(ctx.sync_status(), "timed steps")
    kt = ctx.profile_read()
    ctx.profile(False)
    st = out.stats_dict()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_step = total_ms / args.steps
    # every step traces the same workload (refill keeps the segment budget N x M; the
    # shadow rays vary by a fraction of a percent with the key): the last step's count
    work = float(st["segments"] + st["shadow_rays"])
    rank_work = work * args.steps
    if ws > 1:
        total_ms, all_work = reduce_over_ranks(total_ms, rank_work, "cuda")
    else:
        all_work = rank_work
    value = all_work / (total_ms / 1000.0)
    launches = sum(v[0] for v in kt.values())

    # visit counts for the algorithmic work of the dominant kernel (untimed run, same key)
    p = base.c()
    p.seed = scenes.PHILOX_KEY_BASE + args.warmup + args.steps - 1
    p.flags |= rpr.RP_FLAG_COUNT_VISITS
    rpr.check(ctx.lib.rp_trace(scene.h, ctypes.byref(p), rpr._ptr(lis_d), rpr._ptr(src_d), S,
                               rpr._ptr(out.H), rpr._ptr(out.direct), rpr._ptr(out.stats), None), "count")
    rpr.check(ctx.sync_status(), "count")
    stc = out.stats_dict()

    # e2e: the public host-buffer entry point, H2D of positions and D2H of H + parameters
    e2e_total, e2e_steps = 0.0, 0
    Hh = torch.empty((S, B, K, T), dtype=torch.float32).pin_memory().numpy()
    lis_h = torch.tensor(sc.listener).pin_memory().numpy()
    src_h = torch.tensor(sc.sources).pin_memory().numpy()
    e2e_p = rpr.TraceParams(**WORKLOAD, flags=flags & ~rpr.RP_FLAG_DEVICE_POSITIONS, scene_id=rank)
    if not args.no_e2e:
        e2e_p.seed = scenes.PHILOX_KEY_BASE + 100
        rpr.update(scene, e2e_p, e2e_p.ir_rate_hz, lis_h, src_h, H_host=Hh, want=("H", "params", "stats"))
        e2e_steps = min(args.steps, 3 if args.workload == "large" else 10)
        for i in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            ta = time.perf_counter()
            e2e_p.seed = scenes.PHILOX_KEY_BASE + 200 + i
            res = rpr.update(scene, e2e_p, e2e_p.ir_rate_hz, lis_h, src_h, H_host=Hh, want=("H", "params", "stats"))
            e2e_total += time.perf_counter() - ta
    e2e_work = float(res["stats"]["segments"] + res["stats"]["shadow_rays"]) if e2e_steps else 0.0
    e2e_value = e2e_work * e2e_steps / e2e_total * (ws if ws > 1 else 1) if e2e_total > 0 else None
    h2d = (S + 1) * 3 * 4
    d2h = Hh.nbytes + S * B * C_sizeof("rp_reverb_params") + C_sizeof("rp_trace_stats")

    if rank != 0:
        return 0
    clocks = clk.summary()
    # roofline of the dominant kernel: BVH traversal is bound by the ALU pipe, not HBM
    name = max(kt, key=lambda k: kt[k][1])
    n_l, tot = kt[name]
    # the kernel's time per update: an update may launch it once per record chunk
    # (chunks past the update's work return at once), so the work of one update is
    # set against all of its launches in that update
    avg_s = tot / args.steps / 1000.0
    idx = 1 if name == "shadow" else 0
    ops = stc["node_visits"][idx] * ALU_OPS_PER_NODE + stc["tri_tests"][idx] * ALU_OPS_PER_TRI
    fops = stc["node_visits"][idx] * FMA_OPS_PER_NODE + stc["tri_tests"][idx] * FMA_OPS_PER_TRI
    achieved = ops / avg_s / 1e12
    peak = minmax_peak / 1e12
    dram = NCU_SHADOW_DRAM.get(args.workload)
    traffic = (dram[0] * st["shadow_rays"] / dram[1]
               if dram and name == "shadow" and not args.fp32_paths and args.shadow_mode != "lanes" else None)
    shares = {k: round(v[1] / sum(x[1] for x in kt.values()), 4) for k, v in kt.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.fp32_paths else "f32+f64path",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "triangles": sc.num_tris, "sources": S, "bands": B,
                   "rays": WORKLOAD["num_rays"], "max_order": WORKLOAD["max_order"], "bins": T, "sh_coeffs": K,
                   "budget_refill": int(WORKLOAD.get("budget_refill", 0)),
                   "path_precision": "fp32" if args.fp32_paths else "fp64 path state, fp32 traversal",
                   "shadow_rays": args.shadow_mode,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{ws}"},
        "updates_per_s": ws * 1000.0 / ms_step,
        "closest_hit_segments_per_step": st["segments"], "shadow_rays_per_step": st["shadow_rays"],
        "primaries_per_step": st["primaries"], "refill_waves": st["waves"],
        "bvh": {"build_ms": round(float(info.build_ms), 2), "max_depth": int(info.max_depth),
                "nodes": int(info.num_nodes),
                "node_visits_per_segment": stc["node_visits"][0] / max(1, stc["segments"]),
                "node_visits_per_shadow_ray": stc["node_visits"][1] / max(1, stc["shadow_rays"]),
                "tri_tests_per_segment": stc["tri_tests"][0] / max(1, stc["segments"]),
                "tri_tests_per_shadow_ray": stc["tri_tests"][1] / max(1, stc["shadow_rays"]),
                "shadow_items": stc["hits_stored"] * S,
                "packet_walks": stc["packet_walks"],
                "rays_per_packet_walk": stc["shadow_rays"] / max(1, stc["packet_walks"]),
                "node_fetches_per_packet_walk": stc["packet_steps"] / max(1, stc["packet_walks"])},
        "roofline": {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_note": ("DRAM bytes per update of the shadow-ray kernel, from an ncu capture at "
                                      "fewer primaries scaled by shadow rays") if traffic else None,
                     "launches_per_update": n_l / args.steps,
                     "peak_note": "FP32 min/max instructions per second, measured on this GPU by "
                                  "rp_measure_pipe_peaks (independent chains on every SM, CUDA events)",
                     "algorithmic": f"{ALU_OPS_PER_NODE:.0f} FP32 min/max/compare per node visit + "
                                    f"{ALU_OPS_PER_TRI:.0f} compares per triangle test, visits counted on the "
                                    f"same update",
                     "fma_pipe": {"achieved": fops / avg_s / 1e12, "peak": fma_peak / 1e12,
                                  "frac": fops / avg_s / fma_peak, "unit": "T FMA-pipe instructions/s",
                                  "algorithmic": f"{FMA_OPS_PER_NODE:.0f} per node visit + "
                                                 f"{FMA_OPS_PER_TRI:.0f} per triangle test"}},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in kt.items()},
        "kernel_share": shares,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": 1000 * e2e_total / e2e_steps if e2e_total > 0 else None, "steps": e2e_steps},
        "clocks": clocks,
    }
    issue = issue_roofline(args.workload if not args.fp32_paths and args.shadow_mode != "lanes" else "",
                           name, float(st["shadow_rays"]), avg_s,
                           torch.cuda.get_device_properties(0).multi_processor_count,
                           clocks.get("sm_mhz") or clocks.get("sm_max_mhz"))
    if issue:
        line["roofline"]["issue"] = issue
    if cpu:
        line["cpu_baseline"] = cpu
    if ws == 1 and not args.no_learned:
        line["updates_per_s_at_5pct_decay_err"] = learned_at_bar(ctx)
    print(json.dumps(line), flush=True)
    return 0


def C_sizeof(name):
    import ctypes
    from paper_1803_00430_gb300 import rpr
    return ctypes.sizeof(getattr(rpr, name))


if __name__ == "__main__":
    sys.exit(main())
