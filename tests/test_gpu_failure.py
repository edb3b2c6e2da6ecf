"""Failure detection without a GPU fault.

Every traversal query has an iteration cap, every internal buffer a capacity; each
ends its work and records an RP_ERR_* code in the device status word, which
rp_sync_status returns after the stream is synchronised.  These tests make them
fire through the context's debug limits (a traversal cap of a few node visits, a
few stored-reflection or record slots), check the code that comes back, and check
that the next call with the normal limits runs normally and matches the oracle.

The bounds-checked build (RP_CHECKED: every reflection, record, key, cell and
histogram index is tested before use) runs the tiny shoebox against the oracle in a
child process, since a process loads one build of the library."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1803_00430_gb300 import rpr, scenes  # noqa: E402

import parity_util as pu  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

TINY = dict(num_rays=4000, max_order=20, sh_order=1, num_bins=1000, min_order=1, ir_rate_hz=1000.0,
            seed=scenes.PHILOX_KEY_BASE + 5)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00430_gb300 import build
    build.build()
    c = rpr.Context(0)
    yield c
    c.set_debug_limits()
    c.close()


def _trace_expect(ctx, scene, sc, p, code):
    out = rpr.trace(scene, p, sc.listener, sc.sources, sync=False)
    st = ctx.sync_status()
    assert st == rpr.RP_ERR[code], rpr.STATUS.get(st, st)
    assert out.stats_dict()["error"] == rpr.RP_ERR[code]
    # the status word was cleared by the read
    assert ctx.sync_status() == rpr.RP_OK
    return out


def _normal_call_matches_oracle(ctx, scene, sc, p):
    g = pu.run_gpu(ctx, sc, p, scene=scene)
    assert g["stats"]["error"] == 0
    o = pu.run_oracle(sc, p)
    pu.assert_parity(g, o, p.num_rays)


def test_tiny_iteration_cap_times_out_without_hang_then_recovers(ctx):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    assert scene.info().num_nodes > 3
    p = rpr.TraceParams(**TINY)
    for mode in (0, rpr.RP_FLAG_SHADOW_LANES):  # the packet walk and the resumable one-ray walk
        ctx.set_debug_limits(iter_cap=2)
        q = rpr.TraceParams(**{**TINY, "flags": mode})
        _trace_expect(ctx, scene, sc, q, "RP_ERR_TIMEOUT")
    ctx.set_debug_limits()
    _normal_call_matches_oracle(ctx, scene, sc, p)


def test_too_small_reflection_capacity_then_retry(ctx):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(**TINY)
    ctx.set_debug_limits(hit_cap=1000)
    out = _trace_expect(ctx, scene, sc, p, "RP_ERR_CAPACITY")
    assert out.stats_dict()["hits_stored"] == 1000  # the slots that existed were filled, no more
    ctx.set_debug_limits()
    _normal_call_matches_oracle(ctx, scene, sc, p)


def test_too_small_record_capacity_then_retry(ctx):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(**TINY)
    ctx.set_debug_limits(record_cap=500)
    _trace_expect(ctx, scene, sc, p, "RP_ERR_CAPACITY")
    ctx.set_debug_limits()
    _normal_call_matches_oracle(ctx, scene, sc, p)


def test_negative_limit_is_rejected(ctx):
    lim = rpr.rp_debug_limits(-1, 0, 0, 0)
    import ctypes
    assert ctx.lib.rp_set_debug_limits(ctx.h, ctypes.byref(lim)) == rpr.RP_ERR["RP_ERR_INVALID_ARG"]


CHECKED_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_1803_00430_gb300 import build, rpr, scenes
build.build(checked=True)
assert rpr.library_path().endswith("checked/librpr.so"), rpr.library_path()
import parity_util as pu
ctx = rpr.Context(0)
for sc, p in ((scenes.shoebox(num_sources=2),
               rpr.TraceParams(num_rays=4000, max_order=20, sh_order=1, num_bins=1000, seed=7)),
              (scenes.shoebox(bands=8, num_sources=3),
               rpr.TraceParams(num_rays=2000, max_order=12, sh_order=3, num_bins=300, min_order=0, seed=8,
                               flags=rpr.RP_FLAG_SHADOW_LANES))):
    g = pu.run_gpu(ctx, sc, p)
    assert g["stats"]["error"] == 0, g["stats"]["error"]
    o = pu.run_oracle(sc, p)
    rep = pu.assert_parity(g, o, p.num_rays, check_params=False)
    print("checked build parity", rep)
print("CHECKED_OK")
"""


def test_bounds_checked_build_on_the_tiny_shoebox(ctx):
    env = dict(os.environ, RPR_CHECKED="1")
    code = CHECKED_SCRIPT.format(root=ROOT, tests=HERE)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
