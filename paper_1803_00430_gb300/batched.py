"""Batched form of the update: many scenes of uneven size, source count and ray
budget traced and estimated in the same persistent launches (rp_batch_*), replayed
as a CUDA graph with autotuned launch shapes, timed against the plain form -- one
rp_trace + rp_estimate per scene -- on the same scenes, rays and Philox keys.

    python -m paper_1803_00430_gb300.batched [--scenes 512] [--steps 3] [--warmup 1]

Prints one JSON object.  Both forms run the same algorithm on the same random
numbers, so they trace the same segments and shadow rays; the timed work per step
is taken from the batch's statistics.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import rpr, scenes

TRACE = dict(max_order=64, sh_order=2, num_bins=2000, min_order=1, ir_rate_hz=1000.0)
# the large workload's update (procedural city): 1M primaries x 200 reflections per listener
CITY_TRACE = dict(max_order=200, sh_order=3, num_bins=3000, min_order=1, ir_rate_hz=1000.0)
CITY_RAYS = 1_000_000


def build(ctx: rpr.Context, n_scenes: int, bands: int = 8):
    """The batched workload's scenes (procedural rooms and corridors, sizes from
    scenes.batched_specs): (Scene handles, scene descriptions, ray counts)."""
    specs = scenes.batched_specs(n_scenes=n_scenes, bands=bands)
    scs = [scenes.room_or_corridor(sd, tris, bands=bands, num_sources=S) for sd, tris, S, _ in specs]
    rs = [rpr.Scene.from_scene(ctx, sc) for sc in scs]
    return rs, scs, [r for *_, r in specs]


def build_city(ctx: rpr.Context, n_listeners: int):
    """The large workload as a batch: the city's one BVH, its 256 sources, and
    n_listeners listeners (one update each, 1M primaries x 200 reflections)."""
    import dataclasses
    city = scenes.city()
    r = rpr.Scene.from_scene(ctx, city)
    scs = [dataclasses.replace(city, listener=l) for l in scenes.city_listeners(city, n_listeners)]
    return [r] * len(scs), scs, [CITY_RAYS] * len(scs)


def _events_ms(fn, steps: int, flush) -> float:
    """Mean milliseconds per call of fn over `steps` calls, CUDA events on the
    current stream, L2 flushed before each call (outside the events)."""
    import torch
    st = torch.cuda.current_stream()
    total = 0.0
    for i in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn(i)
        b.record(st)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    return total / steps


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--scenes", type=int, default=512)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--autotune-cache", default="", help="text file of autotuned launch shapes ('' = none)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-scene plain form")
    ap.add_argument("--city", type=int, default=0, metavar="K",
                    help="the large workload instead: the city with K listeners (1M primaries x 200 reflections each)")
    ap.add_argument("--shadow-mode", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="shadow rays: 1 packets, 2 one per lane, 0 the default (packets); -1 autotunes")
    a = ap.parse_args(argv)
    t_setup = time.time()
    ctx = rpr.Context(0, torch.cuda.current_stream())
    trace = CITY_TRACE if a.city else TRACE
    rs, scs, rays = build_city(ctx, a.city) if a.city else build(ctx, a.scenes)
    p = rpr.TraceParams(**trace)
    items = [(rs[i], scs[i].listener, scs[i].sources, rays[i], i) for i in range(len(rs))]
    b = rpr.Batch(ctx, items, p)
    info = b.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    setup_s = time.time() - t_setup
    tune_ms = None
    if a.shadow_mode >= 0:
        t = b.tuning()
        t.shadow_mode = a.shadow_mode
        b.set_tuning(t)
    elif not a.no_autotune:
        t, tune_ms = b.autotune(seed=scenes.PHILOX_KEY_BASE, cache_path=a.autotune_cache or None)
    tuning = b.tuning()
    for w in range(a.warmup):
        b.run(seed=scenes.PHILOX_KEY_BASE + 1 + w, use_graph=True)

    def batched_step(i):
        b.run(seed=scenes.PHILOX_KEY_BASE + 100 + i, use_graph=True, sync=False)

    ms_batched = _events_ms(batched_step, a.steps, flush)
    rpr.check(ctx.sync_status(), "batched steps")
    st = b.stats_dict()
    work = float(st["segments"] + st["shadow_rays"])
    out = {
        "form": "batched", "workload": f"city x {a.city} listeners" if a.city else "rooms and corridors",
        "scenes": len(rs), "total_sources": b.S, "total_rays": int(info.total_rays),
        "groups": int(info.num_groups), "triangles_total": int(sum(len(sc.tris) for sc in {id(r): sc for r, sc in zip(rs, scs)}.values())),
        "ms_per_step": ms_batched, "updates_per_s": len(rs) * 1000.0 / ms_batched,
        "ray_segments_per_s": work * 1000.0 / ms_batched,
        "segments_per_step": st["segments"], "shadow_rays_per_step": st["shadow_rays"],
        "tuning": {"chunk_rays": tuning.chunk_rays, "shadow_steps": tuning.shadow_steps,
                   "paths_blocks_per_sm": tuning.paths_blocks_per_sm,
                   "shadow_blocks_per_sm": tuning.shadow_blocks_per_sm, "shadow_mode": tuning.shadow_mode},
        "autotune_best_ms": tune_ms, "setup_s": round(setup_s, 1),
        "l2": "flushed between timed steps (256 MiB write)",
    }
    if not a.no_plain:
        # the plain form: one trace + estimate per scene, in the same order, same keys
        S_max = max(sc.num_sources for sc in scs)
        K, T, B = p.K, p.num_bins, rs[0].B
        H = torch.empty((S_max, B, K, T), dtype=torch.float32, device="cuda")
        direct = torch.zeros(S_max * rpr.C.sizeof(rpr.rp_direct), dtype=torch.uint8, device="cuda")
        stats = torch.zeros(rpr.C.sizeof(rpr.rp_trace_stats), dtype=torch.uint8, device="cuda")
        params = torch.empty(S_max * B * rpr.C.sizeof(rpr.rp_reverb_params), dtype=torch.uint8, device="cuda")
        pos = [(torch.tensor(sc.listener, device="cuda"), torch.tensor(sc.sources, device="cuda")) for sc in scs]
        ep = rpr.rp_estimate_params(p.ir_rate_hz, 0.0, 0.0)
        for i, r in enumerate(rs):  # size the workspace once, outside the timed region
            q = rpr.TraceParams(**trace, num_rays=rays[i], scene_id=i)
            rpr.check(ctx.lib.rp_trace_reserve(r.h, rpr.C.byref(q.c()), scs[i].num_sources), "reserve")

        def plain_step(k):
            for i, r in enumerate(rs):
                q = rpr.TraceParams(**trace, num_rays=rays[i], scene_id=i,
                                    seed=scenes.PHILOX_KEY_BASE + 100 + k, flags=rpr.RP_FLAG_DEVICE_POSITIONS)
                S = scs[i].num_sources
                rpr.check(ctx.lib.rp_trace(r.h, rpr.C.byref(q.c()), rpr._ptr(pos[i][0]), rpr._ptr(pos[i][1]), S,
                                           rpr._ptr(H), rpr._ptr(direct), rpr._ptr(stats), None), "rp_trace")
                rpr.check(ctx.lib.rp_estimate(ctx.h, rpr._ptr(H), rpr._ptr(direct), S, B, K, T, rpr.C.byref(ep),
                                              rpr._ptr(params), None), "rp_estimate")

        plain_step(0)
        torch.cuda.synchronize()
        ms_plain = _events_ms(plain_step, max(1, min(a.steps, 2)), flush)
        rpr.check(ctx.sync_status(), "plain steps")
        out["plain"] = {"ms_per_step": ms_plain, "updates_per_s": len(rs) * 1000.0 / ms_plain,
                        "ray_segments_per_s": work * 1000.0 / ms_plain}
        out["speedup_vs_plain"] = ms_plain / ms_batched
    print(json.dumps(out))
    b.close()
    ctx.close()


if __name__ == "__main__":
    main()
