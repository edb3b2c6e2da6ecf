"""Pins of the oracle's temporal coherence (Section 5): early-reflection paths, the
diffuse path cache, the prioritisation of early paths and the impulse-response cache.

  * Early paths against the already pinned histogram: with fully diffuse surfaces (no
    specular bounce, so no source-sphere terms) the histogram traced with min_order = 1
    minus the one traced with min_order = m holds exactly the diffuse rain of orders
    1 .. m-1, so the early paths of the min_order = m step must add up to that
    difference, coefficient by coefficient (same random numbers; FP64 rounding only).
  * A path of one record carries the SH basis of its arrival direction.
  * Exponential smoothing: a constant input is a fixed point; a step is followed by
    1 - (1 - alpha)^n and reaches 1 - 1/e after tau seconds of updates; alpha = 1 on
    the first update.
  * Prioritisation: the rendered paths are the n_er largest by total energy (checked
    against a brute-force sort), and rendered + spilled + discarded energy is the
    cache's total; the spill adds exactly the spilled paths' SH energy to the IR.
"""
import numpy as np
import pytest

import oracle
from paper_1803_00430_gb300 import scenes


def _diffuse_box(num_sources=2, bands=4):
    return scenes.shoebox(num_sources=num_sources, bands=bands, scattering=np.ones(bands))


@pytest.mark.parametrize("min_order", [2, 3])
def test_early_paths_add_up_to_the_histogram_orders_they_take(min_order):
    sc = _diffuse_box()
    osc = oracle.OracleScene.from_scene(sc)
    common = dict(num_rays=3000, max_order=12, sh_order=2, num_bins=4000, ir_rate_hz=1000.0, seed=77)
    H1, st1, _ = oracle.trace(osc, oracle.TraceParams(min_order=1, **common), sc.listener, sc.sources)
    Hm, stm, _ = oracle.trace(osc, oracle.TraceParams(min_order=min_order, **common), sc.listener, sc.sources)
    assert st1["late"].sum() == 0.0 and stm["late"].sum() == 0.0
    p = oracle.TraceParams(min_order=min_order, **common)
    er = oracle.er_paths(osc, p, sc.listener, sc.sources, int(stm["primaries"]))
    assert len(er["source"]) > 0
    assert set(er["order"].tolist()) == set(range(1, min_order))
    assert (er["tri2"][er["order"] == 1] == oracle.ER_NONE).all()
    assert ((er["tri1"] >= 0) & (er["tri1"] < sc.num_tris)).all()
    diff = (H1 - Hm).sum(axis=3)  # [S][B][K]
    tot = np.zeros_like(diff)
    for i in range(len(er["source"])):
        tot[er["source"][i]] += er["sh"][i]
    np.testing.assert_allclose(tot, diff, rtol=1e-10, atol=1e-12 * np.abs(diff).max())
    # the omnidirectional coefficient carries the energy: sh[b][0] = energy[b] / sqrt(4 pi)
    np.testing.assert_allclose(er["sh"][:, :, 0], er["energy"] / np.sqrt(4 * np.pi), rtol=1e-12)
    # delays lie between the direct path's and the longest possible early path's
    assert (er["delay"] > 0).all() and (er["delay"] < 1.0).all()


def test_a_single_record_path_carries_its_arrival_direction():
    sc = _diffuse_box(num_sources=1)
    osc = oracle.OracleScene.from_scene(sc)
    p = oracle.TraceParams(num_rays=40, max_order=4, sh_order=3, num_bins=2000, min_order=2, seed=5)
    rec = oracle.er_records(osc, p, sc.listener, sc.sources, 40)
    er = oracle.er_paths(osc, p, sc.listener, sc.sources, 40)
    keys = {}
    for r in rec:
        keys.setdefault((int(r[0]), int(r[2]), int(r[3])), []).append(r)
    single = [v[0] for v in keys.values() if len(v) == 1]
    assert single
    for r in single:
        i = np.nonzero((er["source"] == int(r[0])) & (er["tri1"] == int(r[2])) & (er["tri2"] == int(r[3])))[0][0]
        # the primary direction of the record's ray, from its Philox draws (Section 5's
        # uniform sphere: z = 1 - 2 u0, phi = 2 pi u1, top 24 bits)
        x = oracle.philox4x32_10([int(r[5]), p.scene_id, 0, 0], [p.seed & 0xFFFFFFFF, p.seed >> 32])
        u0, u1 = (int(x[0]) >> 8) / 2.0 ** 24, (int(x[1]) >> 8) / 2.0 ** 24
        z = 1 - 2 * u0
        d = np.array([np.sqrt(1 - z * z) * np.cos(2 * np.pi * u1), np.sqrt(1 - z * z) * np.sin(2 * np.pi * u1), z])
        Y = oracle.sh_eval(3, d)
        np.testing.assert_allclose(er["sh"][i], er["energy"][i][:, None] * Y[None, :], rtol=1e-9, atol=1e-15)
        assert er["delay"][i] == pytest.approx(r[4] / p.speed_of_sound, rel=1e-12)


def _paths(keys, E, delay, B=2, K=4, rng=None):
    rng = rng or np.random.default_rng(0)
    n = len(keys)
    sh = np.zeros((n, B, K))
    sh[:, :, 0] = np.asarray(E) / np.sqrt(4 * np.pi)
    sh[:, :, 1:] = rng.normal(scale=0.01, size=(n, B, K - 1))
    return {"source": np.array([k[0] for k in keys]), "tri1": np.array([k[1] for k in keys]),
            "tri2": np.array([k[2] for k in keys]), "order": np.array([1 if k[2] < 0 else 2 for k in keys]),
            "energy": np.asarray(E, float).reshape(n, B), "sh": sh, "delay": np.asarray(delay, float)}


def test_smoothing_alpha_and_ir_cache_step_response():
    assert oracle.smoothing_alpha(0.1, 3.0, True) == 1.0
    assert oracle.smoothing_alpha(0.1, 0.0, False) == 1.0
    dt, tau = 0.05, 3.0
    a = oracle.smoothing_alpha(dt, tau, False)
    assert a == pytest.approx(1 - np.exp(-dt / tau))
    L = np.random.default_rng(1).uniform(size=(2, 3, 4, 10))
    C = oracle.ir_cache_update(None, L, 1.0)
    for _ in range(7):
        C = oracle.ir_cache_update(C, L, a)
    np.testing.assert_allclose(C, L, rtol=1e-14)  # a constant IR is a fixed point
    C = np.zeros_like(L)
    n = int(round(tau / dt))
    for _ in range(n):
        C = oracle.ir_cache_update(C, L, a)
    np.testing.assert_allclose(C, (1 - np.exp(-1.0)) * L, rtol=1e-12)  # tau seconds: 1 - 1/e of the step


def test_path_cache_fixed_point_decay_and_delay_weighting():
    a = 0.2
    f1 = _paths([(0, 3, -1), (1, 4, 7)], [[1.0, 2.0], [0.5, 0.5]], [0.010, 0.020])
    c = oracle.er_cache_update(None, f1, 1.0)
    for _ in range(5):
        c = oracle.er_cache_update(c, f1, a)
    np.testing.assert_allclose(c["energy"], f1["energy"], rtol=1e-14)
    np.testing.assert_allclose(c["sh"], f1["sh"], rtol=1e-13)
    np.testing.assert_allclose(c["delay"], f1["delay"], rtol=1e-14)
    # a path no longer found decays as (1 - alpha)^n; a new path enters with alpha
    f2 = _paths([(1, 4, 7), (2, 5, -1)], [[0.5, 0.5], [4.0, 4.0]], [0.020, 0.030])
    c2 = oracle.er_cache_update(c, f2, a)
    c3 = oracle.er_cache_update(c2, f2, a)
    i0 = np.nonzero(c3["source"] == 0)[0][0]
    np.testing.assert_allclose(c3["energy"][i0], (1 - a) ** 2 * f1["energy"][0], rtol=1e-13)
    i2 = np.nonzero(c2["source"] == 2)[0][0]
    np.testing.assert_allclose(c2["energy"][i2], a * f2["energy"][1], rtol=1e-13)
    # the same key at two delays: energy-weighted mean
    g = _paths([(0, 3, -1)], [[1.0, 1.0]], [0.050])
    c4 = oracle.er_cache_update(oracle.er_cache_update(None, f1, 1.0), g, 0.5)
    i = np.nonzero(c4["source"] == 0)[0][0]
    w1, w2 = 0.5 * 3.0, 0.5 * 2.0
    assert c4["delay"][i] == pytest.approx((w1 * 0.010 + w2 * 0.050) / (w1 + w2), rel=1e-14)
    # pruning drops paths whose energy fell to the threshold (totals 3 and 1 times 0.01)
    c5 = oracle.er_cache_update(c, _paths([], np.zeros((0, 2)), []), 0.99, prune=0.05)
    assert len(c5["source"]) == 0


def test_prioritisation_and_spill_conserve_energy():
    rng = np.random.default_rng(3)
    n, B, K = 300, 2, 4
    keys = [(int(rng.integers(0, 3)), int(t), -1) for t in rng.permutation(5000)[:n]]
    E = rng.exponential(size=(n, B))
    E[:7] = 0.0  # below any threshold
    c = oracle.er_cache_update(None, _paths(keys, E, rng.uniform(0.001, 0.2, n), B, K, rng), 1.0)
    top, rest = oracle.er_prioritize(c, n_er=100, hearing_threshold=1e-12)
    inten = c["energy"].sum(axis=1)
    brute = np.argsort(-inten, kind="stable")[:100]
    assert set(top.tolist()) == set(brute.tolist())
    assert (np.diff(inten[top]) <= 0).all()
    dropped = np.setdiff1d(np.arange(len(inten)), np.concatenate([top, rest]))
    assert (inten[dropped] <= 1e-12).all()
    assert inten[top].sum() + inten[rest].sum() + inten[dropped].sum() == pytest.approx(inten.sum(), rel=1e-14)
    H = np.zeros((3, B, K, 300))
    H2 = oracle.er_spill(H, c, rest, 1000.0)
    spilled = np.zeros((3, B, K))
    for i in rest:
        if np.floor(c["delay"][i] * 1000.0) < 300:
            spilled[c["source"][i]] += c["sh"][i]
    np.testing.assert_allclose(H2.sum(axis=3), spilled, rtol=1e-12, atol=1e-15)
