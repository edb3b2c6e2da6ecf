"""The budget refill's planner (Sec. 4.1's refill of unused segments): store passes
against counting passes.

A store pass traces candidate rays once and keeps their reflections, records and
statistics; candidates past the planned waves are dropped afterwards.  The counting
passes (rp_set_debug_limits spec_slots = -1) trace the planned rays a second time.
Both plan the same waves over the same ray ids, so every count agrees exactly, the
double sums agree to their summation order and the histograms to the order in which
records reach a bin.  Covered: waves that end inside the first pass (dropped
candidates), waves that reach past it (a second pass with its speculative tail), the
paper's setting (min order 3, IR at 100 Hz), and a store pass with a single
speculative slot, which gives up and falls back to counting passes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1803_00430_gb300 import build, rpr, scenes  # noqa: E402
import parity_util as pu  # noqa: E402

INT_KEYS = ("segments", "shadow_rays", "primaries", "waves", "contributions", "sphere_hits", "hits_stored",
            "mfp_count", "mfp_count_np", "fp64_reruns", "error")
SUM_KEYS = ("escaped", "absorbed", "remaining", "late", "mfp_sum", "mfp_sum_np")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = rpr.Context(0)
    yield c
    c.close()


def _open_floor():
    # a floor and one wall: most rays escape after a reflection or two, so the waves
    # reach far past the first pass's 4 N candidates
    v = np.array([[-20, -20, 0], [20, -20, 0], [20, 20, 0], [-20, 20, 0],
                  [5, -20, 0], [5, 20, 0], [5, 20, 10], [5, -20, 10]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    return scenes.Scene("open", v, t, np.zeros(4, np.int32), np.full((1, 2), 0.1, np.float32),
                        np.full((1, 2), 0.5, np.float32), np.array([0.0, 0.0, 1.5], np.float32),
                        np.array([[2.0, 1.0, 1.5], [-3.0, 2.0, 1.0]], np.float32))


def _open_box(sources=2):
    # a shoebox with one wall missing: the waves end inside the first pass
    sc = scenes.shoebox(num_sources=sources)
    keep = np.ones(len(sc.tris), dtype=bool)
    keep[:2] = False
    sc.tris, sc.tri_material = sc.tris[keep], sc.tri_material[keep]
    return sc


def _run(ctx, scene, sc, p, spec_slots):
    ctx.set_debug_limits(spec_slots=spec_slots)
    try:
        ctx.profile(True)
        ctx.profile_reset()
        out = rpr.trace(scene, p, sc.listener, sc.sources)
        torch.cuda.synchronize()
        paths = ctx.profile_read().get("paths", (0, 0.0))[0]
        ctx.profile(False)
    finally:
        ctx.set_debug_limits()
    return out, paths


def _same(a, b):
    sa, sb = a.stats_dict(), b.stats_dict()
    for k in INT_KEYS:
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    for k in SUM_KEYS:
        np.testing.assert_allclose(sa[k], sb[k], rtol=1e-9, atol=1e-12, err_msg=k)
    Ha, Hb = a.H.double().cpu().numpy(), b.H.double().cpu().numpy()
    assert np.abs(Hb).max() > 0
    np.testing.assert_allclose(Ha, Hb, rtol=0, atol=1e-6 * np.abs(Hb).max())
    da, db = a.direct_dict(), b.direct_dict()
    for k in da:
        np.testing.assert_array_equal(da[k], db[k], err_msg=k)


CASES = {
    "waves_past_the_first_pass": (_open_floor, dict(num_rays=3000, max_order=50, sh_order=1, num_bins=400,
                                                    budget_refill=1, seed=scenes.PHILOX_KEY_BASE + 71)),
    "waves_inside_the_first_pass": (_open_box, dict(num_rays=3000, max_order=20, sh_order=1, num_bins=800,
                                                    budget_refill=1, seed=scenes.PHILOX_KEY_BASE + 72)),
    "paper_setting": (lambda: _open_box(3), dict(num_rays=50, max_order=200, sh_order=1, num_bins=300,
                                                 min_order=3, ir_rate_hz=100.0, budget_refill=1,
                                                 seed=scenes.PHILOX_KEY_BASE + 73)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_store_passes_match_counting_passes(ctx, case):
    make, kw = CASES[case]
    sc = make()
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(**kw)
    st, n_store = _run(ctx, scene, sc, p, 0)
    ct, n_count = _run(ctx, scene, sc, p, -1)
    s = st.stats_dict()
    assert s["error"] == 0 and s["waves"] > 1
    _same(st, ct)
    # the counting passes trace the planned rays once more
    assert n_count == n_store + 1
    if case != "waves_past_the_first_pass":
        assert n_store == 1  # the waves end inside the first pass: one launch of the paths kernel
    else:
        assert s["primaries"] > 4 * p.num_rays and n_store >= 2
    scene.close()


def test_store_pass_with_one_slot_falls_back(ctx):
    # one speculative slot: the second pass takes almost all of its candidates as
    # inside the waves, the waves end before them, and the step is traced again with
    # counting passes
    sc = _open_floor()
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=2000, max_order=40, sh_order=1, num_bins=400, budget_refill=1,
                        seed=scenes.PHILOX_KEY_BASE + 74)
    fb, n_fb = _run(ctx, scene, sc, p, 1)
    ct, n_count = _run(ctx, scene, sc, p, -1)
    _same(fb, ct)
    assert n_fb > n_count  # the store passes, then the counting passes and the planned rays
    # the context is left as it was: the next call plans with store passes
    st, n_store = _run(ctx, scene, sc, p, 0)
    _same(st, ct)
    assert n_store < n_count
    scene.close()


def test_store_passes_match_the_oracle_waves(ctx):
    # the waves the store passes keep are the oracle's (Sec. 4.1: each later wave takes
    # floor(unused budget / M) new primaries)
    make, kw = CASES["waves_inside_the_first_pass"]
    sc = make()
    p = rpr.TraceParams(**{**kw, "num_rays": 1500})
    g = pu.run_gpu(ctx, sc, p, want_hash=False)
    o = pu.run_oracle(sc, p, want_hash=False)
    sg, so = g["stats"], o["stats"]
    for k in ("waves", "primaries", "segments", "mfp_count", "mfp_count_np"):
        assert sg[k] == so[k], k
    np.testing.assert_allclose(sg["mfp_sum"], so["mfp_sum"], rtol=1e-9)
    l1_0, _ = pu.band_l1(g["H"], o["H"])
    assert l1_0.max() <= 1e-3
    g["scene"].close()
