"""Reverberator parameters on the GPU (rp_reverb_configure) against the FP64 oracle
(Sections 4.1 and 4.2): comb delays and their redraw rule over updates, comb gains,
comb input directions and SH gains, the combs' rotations and SH rotation matrices
(recurrence on the GPU, the integral definition in the oracle), and the directional
loudness matrices -- on the same IR and estimated parameters, then end to end."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import reverb as oreverb  # noqa: E402
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


def _compare(g, o, K):
    np.testing.assert_allclose(g["t_comb"], o["t_comb"], rtol=1e-12)
    np.testing.assert_allclose(g["g_comb"], o["g_comb"], rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(g["dir"], o["dir"], atol=1e-6)
    np.testing.assert_allclose(g["comb_in"], o["comb_in"][:, :K], atol=2e-6)
    np.testing.assert_allclose(g["rot"], o["rot"], atol=1e-6)
    np.testing.assert_allclose(g["J"], o["J"], atol=2e-6)
    np.testing.assert_allclose(g["D"], o["D"], atol=2e-5 * max(1.0, np.abs(o["D"]).max()))
    assert g["generation"] == o["generation"] and g["mean_delay"] == pytest.approx(o["mean_delay"], rel=1e-15)


@pytest.mark.parametrize("sh_order", [1, 3])
def test_reverberator_parameters_match_oracle_over_updates(ctx, sh_order):
    sc = scenes.shoebox(num_sources=3)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=8000, max_order=20, sh_order=sh_order, num_bins=1000, min_order=3,
                        seed=scenes.PHILOX_KEY_BASE + 61)
    out = rpr.trace(scene, p, sc.listener, sc.sources)
    prm = rpr.estimate(ctx, out.H, out.direct, p.ir_rate_hz)
    S, B, K = sc.num_sources, sc.num_bands, p.K
    pd = rpr.params_to_dict(prm.cpu().numpy().tobytes(), S, B, K)
    H = out.H.double().cpu().numpy()
    mfp = out.stats_dict()["mean_free_path"]
    rev, ost = None, None
    # the mean free path moving: kept (within 2 sigma), then redrawn
    for u, scale in enumerate([1.0, 1.4, 1.8, 1.82]):
        rev, g = rpr.reverb_configure(ctx, out.H, prm, S, B, K, p.ir_rate_hz, mfp * scale, seed=77, rev=rev)
        o, ost = oreverb.configure(H, pd["rt60_smoothed"], pd["xbar"], mfp * scale, 343.0, p.ir_rate_hz, 77, ost)
        for s in range(S):
            _compare(g[s], o[s], K)
            assert g[s]["resampled"] == o[s]["resampled"]
    assert [o[0]["generation"]] == [2]


def test_reverberator_parameters_end_to_end(ctx):
    """The GPU pipeline (trace, estimate, configure) against the oracle pipeline on
    the oracle's own IR: delays and rotations exactly, directions and gains within
    what the IR's 1e-3 bar allows."""
    sc = scenes.shoebox(num_sources=2)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=20000, max_order=30, sh_order=2, num_bins=1500, min_order=1,
                        seed=scenes.PHILOX_KEY_BASE + 62)
    out = rpr.trace(scene, p, sc.listener, sc.sources)
    prm = rpr.estimate(ctx, out.H, out.direct, p.ir_rate_hz)
    S, B, K = sc.num_sources, sc.num_bands, p.K
    _, g = rpr.reverb_configure(ctx, out.H, prm, S, B, K, p.ir_rate_hz, out.stats_dict()["mean_free_path"], seed=5)
    o = pu.run_oracle(sc, p, want_hash=False)
    oo, _ = oreverb.configure(o["H"], o["params"]["rt60_raw"], o["params"]["xbar"], o["stats"]["mean_free_path"],
                              343.0, p.ir_rate_hz, 5, None)
    for s in range(S):
        np.testing.assert_allclose(g[s]["t_comb"], oo[s]["t_comb"], rtol=1e-5)  # mean free path to 1e-5
        np.testing.assert_allclose(g[s]["J"], oo[s]["J"], atol=2e-6)
        np.testing.assert_allclose(g[s]["g_comb"], oo[s]["g_comb"], rtol=pu.PARAM_BAR)
        assert (np.einsum("ij,ij->i", g[s]["dir"], oo[s]["dir"]) > 0.999).all()
        np.testing.assert_allclose(g[s]["D"], oo[s]["D"], atol=5e-3)
