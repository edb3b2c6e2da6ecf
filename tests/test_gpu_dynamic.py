"""Dynamic scenes: moving objects refitted on the device (rp_scene_refit), and a
moving listener and sources across updates with the estimator's smoothing state.

A refitted scene must answer every query as a scene built from the moved mesh: the
same triangle sequence for every primary ray (64-bit hashes equal) and the same
histogram up to the order in which records reach each bin; both against the FP64
oracle on the moved mesh at the stated bar."""
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


def _move_boxes(sc, first_box, n_boxes, angle, shift):
    """Rigid motion of n_boxes interior boxes of the furnished hall (8 vertices each
    after the hall's own 8): a turn by `angle` about the box's vertical axis, then a
    shift."""
    v = sc.verts.astype(np.float64).copy()
    c, s = np.cos(angle), np.sin(angle)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    for k in range(first_box, first_box + n_boxes):
        sl = slice(8 + 8 * k, 16 + 8 * k)
        ctr = v[sl].mean(axis=0)
        v[sl] = (v[sl] - ctr) @ R.T + ctr + np.asarray(shift)
    out = scenes.Scene(sc.name + "-moved", v.astype(np.float32), sc.tris, sc.tri_material, sc.absorption,
                       sc.scattering, sc.listener, sc.sources)
    return out


def test_refit_answers_as_a_rebuilt_scene_and_the_oracle(ctx):
    sc = scenes.furnished_hall()
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=20000, max_order=64, sh_order=2, num_bins=2000, seed=scenes.PHILOX_KEY_BASE + 9)
    for frame, (angle, shift) in enumerate([(0.35, (0.4, -0.3, 0.0)), (0.7, (0.8, -0.6, 0.2))]):
        moved = _move_boxes(sc, 1500, 500, angle, shift)
        scene.refit(moved.verts)
        info = scene.info()
        assert info.refit_ms > 0
        g = pu.run_gpu(ctx, moved, p, scene=scene)
        fresh = rpr.Scene.from_scene(ctx, moved)
        f = pu.run_gpu(ctx, moved, p, scene=fresh)
        assert abs(fresh.info().ray_epsilon - info.ray_epsilon) <= 1e-7 * fresh.info().ray_epsilon
        np.testing.assert_allclose([info.bounds_lo[k] for k in range(3)], [fresh.info().bounds_lo[k] for k in range(3)])
        assert (g["hash"] == f["hash"]).all()
        assert g["stats"]["segments"] == f["stats"]["segments"]
        assert g["stats"]["shadow_rays"] == f["stats"]["shadow_rays"]
        np.testing.assert_allclose(g["H"], f["H"], rtol=0, atol=1e-6 * np.abs(f["H"]).max())
        o = pu.run_oracle(moved, p)
        rep = pu.assert_parity(g, o, p.num_rays, check_params=False)
        rep.update(pu.assert_well_posed_params(g, o, min_well=64, min_kinds_equal=0.97))
        print(f"frame {frame}: refit {info.refit_ms:.3f} ms (build {fresh.info().build_ms:.3f} ms), {rep}")


def test_refit_rejects_bad_vertices_and_keeps_the_scene(ctx):
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=3000, max_order=10, sh_order=1, num_bins=400, seed=4)
    before = pu.run_gpu(ctx, sc, p, scene=scene)
    bad = sc.verts.copy()
    bad[2, 1] = np.inf
    with pytest.raises(rpr.RprError) as e:
        scene.refit(bad)
    assert e.value.status == rpr.RP_ERR["RP_ERR_NAN_INPUT"]
    with pytest.raises(rpr.RprError) as e:
        scene.refit(sc.verts[:-1])
    assert e.value.status == rpr.RP_ERR["RP_ERR_INVALID_ARG"]
    after = pu.run_gpu(ctx, sc, p, scene=scene)
    assert (before["hash"] == after["hash"]).all()
    # a refit to the same positions changes nothing
    scene.refit(torch.tensor(sc.verts, device="cuda"))
    same = pu.run_gpu(ctx, sc, p, scene=scene)
    assert (before["hash"] == same["hash"]).all()
    np.testing.assert_allclose(same["H"], before["H"], rtol=0, atol=1e-6 * np.abs(before["H"]).max())


def test_moving_listener_and_sources_with_smoothing_state(ctx):
    """Three updates with the listener and sources moving; each update's histogram
    against the oracle at that update's positions, and the RT60 smoothing state
    (alpha = 1 - exp(-dt / tau)) carried across updates as the oracle carries it."""
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    S, B = sc.num_sources, sc.num_bands
    p = rpr.TraceParams(num_rays=10000, max_order=20, sh_order=1, num_bins=1000, seed=scenes.PHILOX_KEY_BASE)
    state = torch.full((S, B), float("nan"), dtype=torch.float64, device="cuda")
    sto = np.full((S, B), np.nan)
    lis0, src0 = sc.listener.copy(), sc.sources.copy()
    for u in range(3):
        step = np.array([0.3, -0.2, 0.1], np.float32) * u
        moved = scenes.Scene(sc.name, sc.verts, sc.tris, sc.tri_material, sc.absorption, sc.scattering,
                             lis0 + step, src0 - step)
        q = rpr.TraceParams(**{**p.__dict__, "seed": p.seed + u})
        out = rpr.trace(scene, q, moved.listener, moved.sources)
        raw = rpr.estimate(ctx, out.H, out.direct, q.ir_rate_hz, dt_update=0.1, tau=3.0, state=state)
        pg = rpr.params_to_dict(raw.cpu().numpy().tobytes(), S, B, q.K)
        o = pu.run_oracle(moved, q, want_hash=False)
        po = oracle.estimate(o["H"], o["direct"]["energy"], q.ir_rate_hz, dt_update=0.1, tau=3.0, state=sto)
        l1, _ = pu.band_l1(out.H.double().cpu().numpy(), o["H"])
        assert l1.max() <= pu.L1_BAR, (u, l1)
        assert (pg["range_kind"] == po["range_kind"]).all()
        np.testing.assert_allclose(pg["rt60_smoothed"], po["rt60_smoothed"], rtol=pu.PARAM_BAR)
        np.testing.assert_allclose(state.cpu().numpy(), sto, rtol=pu.PARAM_BAR)
