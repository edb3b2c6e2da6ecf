"""Timing of the stages that follow the propagation and estimation along the paper's
pipeline: temporal coherence (early-path cache, IR cache), BVH refit for moving
geometry, the reverberator's parameters and the batched SH-domain reverberator.  One
GPU, CUDA events on the context stream around repeated calls, inputs resident in
device memory; prints one JSON object.

    python -m paper_1803_00430_gb300.rows
"""
from __future__ import annotations

import ctypes as C
import json

import numpy as np

from . import rpr, scenes

FS = 48000.0
XO_4 = [176.0, 775.0, 3408.0]                                     # the paper's four bands
XO_8 = [88.4, 176.8, 353.6, 707.1, 1414.2, 2828.4, 5656.9]      # octave bands


def _time_ms(fn, reps: int = 5, warm: int = 2) -> float:
    """Mean device time of fn() over `reps` calls after `warm` calls."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def temporal_coherence(ctx: rpr.Context) -> dict:
    """rp_trace_er against rp_trace on the same update, at the paper's operating point
    (50 primaries x 200 reflections with refill, orders 1-2 early, IR 100 Hz, SH order 1)
    and on the hall (20k primaries, orders 1-2 early); and the IR cache's update of the
    city-sized histogram (256 sources x 8 bands x 16 SH x 3000 bins)."""
    import torch
    out = {}
    cases = {
        "paper_point": (scenes.paper_city(), rpr.TraceParams(num_rays=50, max_order=200, sh_order=1, num_bins=300,
                                                              min_order=3, ir_rate_hz=100.0, budget_refill=1,
                                                              seed=scenes.PHILOX_KEY_BASE + 50)),
        "hall_20k": (scenes.furnished_hall(), rpr.TraceParams(num_rays=20000, max_order=64, sh_order=2, num_bins=2000,
                                                              min_order=3, seed=scenes.PHILOX_KEY_BASE + 51)),
    }
    for name, (sc, p) in cases.items():
        scene = rpr.Scene.from_scene(ctx, sc)
        er = rpr.ERCache(ctx, sc.num_bands, p.sh_order)
        t_er = _time_ms(lambda: er.trace(scene, p, sc.listener, sc.sources, dt_update=0.1, tau_er=1.0))
        t_plain = _time_ms(lambda: rpr.trace(scene, p, sc.listener, sc.sources))
        _, rendered = er.trace(scene, p, sc.listener, sc.sources, dt_update=0.1, tau_er=1.0)
        out[name] = {"triangles": int(sc.tris.shape[0]), "sources": int(sc.sources.shape[0]),
                     "update_with_er_cache_ms": round(t_er, 3), "plain_update_ms": round(t_plain, 3),
                     "cached_paths": int(len(er.read()["source"])), "rendered_paths": int(len(rendered["source"]))}
        er.close()
        scene.close()
    n = 256 * 8 * 16 * 3000
    H = torch.rand(n, device="cuda")
    Cc = torch.zeros(n, device="cuda")
    rpr.ir_cache_update(ctx, H, Cc, 0.1, 3.0, True)
    t = _time_ms(lambda: rpr.ir_cache_update(ctx, H, Cc, 0.1, 3.0, False), reps=20)
    out["ir_cache_city"] = {"cells": n, "ms": round(t, 4), "bytes": 12 * n,
                            "gb_per_s": round(12 * n / (t * 1e-3) / 1e9, 1)}
    return out


def refit(ctx: rpr.Context) -> dict:
    """rp_scene_refit after a rigid move of a block of the city's buildings and of the
    hall's boxes, against a build from scratch."""
    import torch
    out = {}
    for name, sc, block in (("city", scenes.city(), (0, 200_000)), ("hall", scenes.furnished_hall(), (1500, 500))):
        scene = rpr.Scene.from_scene(ctx, sc)
        build_ms = float(scene.info().build_ms)
        v = sc.verts.copy()
        tri = sc.tris
        if name == "hall":
            idx = np.unique(tri[12 + 12 * block[0]:12 + 12 * (block[0] + block[1])].ravel())
        else:
            idx = np.unique(tri[block[0]:block[0] + block[1]].ravel())
        v[idx] += np.array([0.7, -0.4, 0.0], np.float32)
        vd = torch.tensor(v, device="cuda")
        ms = []
        for _ in range(5):
            scene.refit(vd)
            ms.append(float(scene.info().refit_ms))
            scene.refit(torch.tensor(sc.verts, device="cuda"))
        nt = int(tri.shape[0])
        out[name] = {"triangles": nt, "moved_vertices": int(len(idx)), "build_ms": round(build_ms, 3),
                     "refit_ms": round(float(np.median(ms)), 3),
                     # a refit reads the vertices and writes every triangle (48 B) and node (64 B)
                     "written_bytes": 48 * nt + 64 * (nt - 1)}
        scene.close()
    return out


def reverberator(ctx: rpr.Context) -> dict:
    """rp_reverb_configure for 256 sources of the city, and rp_reverb_render of 4096-sample
    blocks at 48 kHz for 256 sources: the paper's four bands at SH order 1, and the city's
    eight octave bands at SH order 3."""
    import torch
    out = {}
    sc = scenes.city()
    scene = rpr.Scene.from_scene(ctx, sc)
    S, B = sc.num_sources, sc.num_bands
    p = rpr.TraceParams(num_rays=20000, max_order=200, sh_order=3, num_bins=3000, budget_refill=1,
                        seed=scenes.PHILOX_KEY_BASE + 60)
    tr = rpr.trace(scene, p, sc.listener, sc.sources)
    prm = rpr.estimate(ctx, tr.H, tr.direct, p.ir_rate_hz)
    mfp = tr.stats_dict()["mean_free_path"]
    rev = torch.zeros(S * C.sizeof(rpr.rp_reverberator), dtype=torch.uint8, device="cuda")

    def configure():
        rpr.check(ctx.lib.rp_reverb_configure(ctx.h, rpr._ptr(tr.H), rpr._ptr(prm), S, B, p.K, p.num_bins,
                                              p.ir_rate_hz, mfp, 343.0, 3, rpr._ptr(rev)), "rp_reverb_configure")
    out["configure_city_256_sources_ms"] = round(_time_ms(configure, reps=10), 3)
    scene.close()
    N = 4096
    audio_ms = 1000.0 * N / FS
    # the paper's setting: 4 bands, SH order 1, parameters from the shoebox repeated
    small = scenes.shoebox(num_sources=1)
    s_scene = rpr.Scene.from_scene(ctx, small)
    ps = rpr.TraceParams(num_rays=6000, max_order=30, sh_order=1, num_bins=1500, min_order=1, seed=61)
    ts = rpr.trace(s_scene, ps, small.listener, small.sources)
    prm_s = rpr.estimate(ctx, ts.H, ts.direct, ps.ir_rate_hz)
    rev_s, _ = rpr.reverb_configure(ctx, ts.H, prm_s, 1, small.num_bands, ps.K, ps.ir_rate_hz,
                                    ts.stats_dict()["mean_free_path"], seed=3)
    cases = (("4_bands_sh1", rev_s.repeat(S), prm_s.repeat(S), small.num_bands, ps.K, XO_4),
             ("8_bands_sh3", rev, prm, B, p.K, XO_8))
    for name, rv, pr, b, k, xo in cases:
        R = rpr.Reverberator(ctx, S, b, k, xo, FS)
        x = torch.randn((S, N), device="cuda") * 0.1
        ctx.profile(True)
        ctx.profile_reset()
        ms = _time_ms(lambda: R.render(rv, pr, x))
        kt = ctx.profile_read()
        ctx.profile(False)
        out[f"render_{name}"] = {"sources": S, "samples": N, "ms_per_block": round(ms, 3),
                                 "real_time_factor": round(audio_ms / ms, 1),
                                 "kernel_ms": {kk: round(v[1] / v[0], 3) for kk, v in kt.items()},
                                 "state_bytes": int(R.state.numel())}
        del R
        torch.cuda.empty_cache()
    s_scene.close()
    return out


def main():
    import torch
    from . import build
    build.build()
    rpr.load()
    ctx = rpr.Context(0, torch.cuda.current_stream())
    res = {"temporal_coherence": temporal_coherence(ctx), "refit": refit(ctx), "reverberator": reverberator(ctx)}
    print(json.dumps(res))
    ctx.close()


if __name__ == "__main__":
    main()
