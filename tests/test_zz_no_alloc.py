"""rp_trace_noalloc: the trace step for callers that must not allocate device memory
during an update -- a real-time audio or game thread that cannot block on the
allocator mid-frame, or an application that owns all device memory through its own
pool.  It takes its temporaries from a fixed static device array instead of
library-allocated workspace.

Checked through the C ABI against rp_trace on the same inputs, on two calls in a
row (the array keeps the previous call's contents, so the second call also checks
that what must start at zero is cleared), with budget refill (rp_trace plans the
refill waves with store passes, rp_trace_noalloc traces them wave by wave: the rays
and results must be the same), plus the size limit.  This file is collected
last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1803_00430_gb300 import build, rpr, scenes  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = rpr.Context(0)
    yield c
    c.close()


def _compare(a, b):
    # same kernels on the same inputs; records reach each bin in run-dependent order
    Ha = a.H.double().cpu().numpy()
    Hb = b.H.double().cpu().numpy()
    np.testing.assert_allclose(Ha, Hb, rtol=0, atol=1e-6 * np.abs(Hb).max())
    sa, sb = a.stats_dict(), b.stats_dict()
    for k in ("segments", "shadow_rays", "primaries", "contributions", "sphere_hits", "hits_stored", "error"):
        assert sa[k] == sb[k], k
    np.testing.assert_allclose(sa["absorbed"], sb["absorbed"], rtol=1e-6)
    da, db = a.direct_dict(), b.direct_dict()
    np.testing.assert_array_equal(da["energy"], db["energy"])


def test_noalloc_matches_rp_trace_on_two_calls_in_a_row(ctx):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p1 = rpr.TraceParams(num_rays=10000, max_order=20, sh_order=1, num_bins=1000, seed=scenes.PHILOX_KEY_BASE)
    p2 = rpr.TraceParams(num_rays=6000, max_order=30, sh_order=2, num_bins=700, min_order=0,
                         seed=scenes.PHILOX_KEY_BASE + 7)
    for p in (p1, p2):
        ref = rpr.trace(scene, p, sc.listener, sc.sources)
        got = rpr.trace_noalloc(scene, p, sc.listener, sc.sources)
        assert got.stats_dict()["error"] == 0
        assert np.abs(got.H.cpu().numpy()).sum() > 0
        _compare(got, ref)


def test_noalloc_matches_rp_trace_with_budget_refill(ctx):
    # an open box (one wall missing) so that rays escape early and the refill waves
    # have unused budget to spend
    sc = scenes.shoebox(num_sources=2)
    keep = np.ones(len(sc.tris), dtype=bool)
    keep[:2] = False
    sc.tris, sc.tri_material = sc.tris[keep], sc.tri_material[keep]
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=3000, max_order=20, sh_order=1, num_bins=800, budget_refill=1,
                        seed=scenes.PHILOX_KEY_BASE + 3)
    ref = rpr.trace(scene, p, sc.listener, sc.sources)
    got = rpr.trace_noalloc(scene, p, sc.listener, sc.sources)
    assert got.stats_dict()["error"] == 0
    assert ref.stats_dict()["waves"] > 1
    assert got.stats_dict()["waves"] == ref.stats_dict()["waves"]
    _compare(got, ref)


def test_noalloc_rejects_problems_beyond_its_scratch(ctx):
    sc = scenes.shoebox()
    scene = rpr.Scene.from_scene(ctx, sc)
    big = rpr.TraceParams(num_rays=2_000_000, max_order=64, sh_order=1, num_bins=1000)
    with pytest.raises(rpr.RprError) as e:
        rpr.trace_noalloc(scene, big, sc.listener, sc.sources)
    assert e.value.status == rpr.RP_ERR["RP_ERR_TOO_LARGE"]
    # the context stays usable
    ok = rpr.trace_noalloc(scene, rpr.TraceParams(num_rays=500, max_order=5, num_bins=200), sc.listener,
                           sc.sources)
    assert ok.stats_dict()["error"] == 0
