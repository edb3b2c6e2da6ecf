"""Temporal coherence on the GPU (rp_trace_er, rp_ir_cache_update) against the FP64
oracle (Section 5): the early-reflection paths of an update and the path cache over
several updates (keys, energy per band, SH directivity, delay), the N_ER rendered
paths, the late IR with the unrendered paths added, and the impulse response cache."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1803_00430_gb300 import rpr, scenes  # noqa: E402

import parity_util as pu  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00430_gb300 import build
    build.build()
    c = rpr.Context(0)
    yield c
    c.close()


def _by_key(d):
    return {(int(d["source"][i]), int(d["tri1"][i]), int(d["tri2"][i])): i for i in range(len(d["source"]))}


def _compare_paths(g, o, rtol=2e-5):
    kg, ko = _by_key(g), _by_key(o)
    assert set(kg) == set(ko), (len(set(kg) - set(ko)), len(set(ko) - set(kg)))
    ig = np.array([kg[k] for k in sorted(ko)])
    io = np.array([ko[k] for k in sorted(ko)])
    np.testing.assert_allclose(g["energy"][ig], o["energy"][io], rtol=rtol, atol=1e-9 * np.abs(o["energy"]).max())
    np.testing.assert_allclose(g["sh"][ig], o["sh"][io], rtol=0, atol=rtol * np.abs(o["sh"]).max())
    np.testing.assert_allclose(g["delay"][ig], o["delay"][io], rtol=1e-6)
    assert (g["order"][ig] == o["order"][io]).all()


def _oracle_update(sc, p, cache, alpha, n_er=100, prune=0.0, thr=0.0):
    o = pu.run_oracle(sc, p, want_hash=False)
    osc = o["scene"]
    frame = oracle.er_paths(osc, pu.oracle_params(p), sc.listener, sc.sources, int(o["stats"]["primaries"]))
    cache = oracle.er_cache_update(cache, frame, alpha, prune=prune)
    top, rest = oracle.er_prioritize(cache, n_er, thr)
    H = oracle.er_spill(o["H"], cache, rest, p.ir_rate_hz)
    return cache, top, H


@pytest.mark.parametrize("min_order", [2, 3])
def test_early_paths_cache_and_rendered_paths_match_oracle(ctx, min_order):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=10000, max_order=20, sh_order=2, num_bins=1000, min_order=min_order,
                        seed=scenes.PHILOX_KEY_BASE + 21)
    er = rpr.ERCache(ctx, sc.num_bands, p.sh_order)
    out, rendered = er.trace(scene, p, sc.listener, sc.sources, n_er=20)
    cache_o, top, Ho = _oracle_update(sc, p, None, 1.0, n_er=20)
    g = er.read()
    assert len(g["source"]) > 20
    _compare_paths(g, cache_o)
    # the rendered paths: the oracle's 20 most intense, in its order
    assert [(int(rendered["source"][i]), int(rendered["tri1"][i]), int(rendered["tri2"][i]))
            for i in range(len(rendered["source"]))] == \
        [(int(cache_o["source"][i]), int(cache_o["tri1"][i]), int(cache_o["tri2"][i])) for i in top]
    # the late IR with the unrendered early paths added
    l1, lk = pu.band_l1(out.H.double().cpu().numpy(), Ho)
    assert l1.max() <= pu.L1_BAR and lk.max() <= 2 * pu.L1_BAR, (l1.max(), lk.max())
    assert out.stats_dict()["error"] == 0


def test_path_cache_and_ir_cache_over_updates(ctx):
    """Three updates 0.1 s apart with tau_ER = 1 s and tau_LR = 3 s: the smoothed path
    cache and the smoothed late IR, with pruning."""
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    er = rpr.ERCache(ctx, sc.num_bands, 1)
    dt, tau_er, tau_lr, prune = 0.1, 1.0, 3.0, 1e-9
    cache_o, C_o = None, None
    C = torch.zeros((sc.num_sources, sc.num_bands, 4, 800), dtype=torch.float32, device="cuda")
    for u in range(3):
        p = rpr.TraceParams(num_rays=6000, max_order=16, sh_order=1, num_bins=800, min_order=3,
                            seed=scenes.PHILOX_KEY_BASE + 40 + u)
        out, _ = er.trace(scene, p, sc.listener, sc.sources, dt_update=dt, tau_er=tau_er, prune=prune, n_er=30)
        a_er = oracle.smoothing_alpha(dt, tau_er, u == 0)
        cache_o, _, Ho = _oracle_update(sc, p, cache_o, a_er, n_er=30, prune=prune)
        _compare_paths(er.read(), cache_o)
        rpr.ir_cache_update(ctx, out.H, C, dt, tau_lr, u == 0)
        C_o = oracle.ir_cache_update(C_o, Ho, oracle.smoothing_alpha(dt, tau_lr, u == 0))
        l1, _ = pu.band_l1(C.double().cpu().numpy(), C_o)
        assert l1.max() <= pu.L1_BAR, (u, l1.max())
    er.reset()
    out, _ = er.trace(scene, p, sc.listener, sc.sources, dt_update=dt, tau_er=tau_er, n_er=30)
    fresh, _, _ = _oracle_update(sc, p, None, 1.0, n_er=30)
    _compare_paths(er.read(), fresh)  # after a reset the cache starts again


def test_early_paths_at_the_papers_operating_point(ctx):
    """Section 5's setting: 50 primaries x 200 reflections with budget refill, orders 1-2
    early, IR 100 Hz, SH order 1, on the city-like scene."""
    sc = scenes.paper_city()
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=50, max_order=200, sh_order=1, num_bins=300, min_order=3, ir_rate_hz=100.0,
                        budget_refill=1, seed=scenes.PHILOX_KEY_BASE + 50)
    er = rpr.ERCache(ctx, sc.num_bands, 1)
    out, rendered = er.trace(scene, p, sc.listener, sc.sources, n_er=100)
    cache_o, top, Ho = _oracle_update(sc, p, None, 1.0, n_er=100)
    _compare_paths(er.read(), cache_o)
    assert len(rendered["source"]) == min(100, len(cache_o["source"]))
    l1, _ = pu.band_l1(out.H.double().cpu().numpy(), Ho)
    assert l1.max() <= pu.L1_BAR
