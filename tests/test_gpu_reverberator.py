"""The SH-domain Schroeder reverberator rendered on the GPU (rp_reverb_render) against
the FP64 oracle (Section 4.1): the same reverberator parameters, a mono input rendered
in blocks of uneven length on the GPU (state carried between them; blocks of 1 and 17
samples leave most crossover chunks empty) and in one
piece by the oracle; plus a batch of many sources for throughput."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import reverberator as orv  # noqa: E402
from paper_1803_00430_gb300 import rpr, scenes  # noqa: E402

XO = [176.0, 775.0, 3408.0]  # the paper's 4 bands


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_00430_gb300 import build
    build.build()
    c = rpr.Context(0)
    yield c
    c.close()


def _setup(ctx, S, sh_order, seed):
    sc = scenes.shoebox(num_sources=S)
    scene = rpr.Scene.from_scene(ctx, sc)
    p = rpr.TraceParams(num_rays=6000, max_order=30, sh_order=sh_order, num_bins=1500, min_order=1,
                        seed=scenes.PHILOX_KEY_BASE + seed)
    out = rpr.trace(scene, p, sc.listener, sc.sources)
    prm = rpr.estimate(ctx, out.H, out.direct, p.ir_rate_hz)
    rev, cfg = rpr.reverb_configure(ctx, out.H, prm, S, sc.num_bands, p.K, p.ir_rate_hz,
                                    out.stats_dict()["mean_free_path"], seed=3)
    pd = rpr.params_to_dict(prm.cpu().numpy().tobytes(), S, sc.num_bands, p.K)
    return sc, p, prm, rev, cfg, pd


@pytest.mark.parametrize("sh_order", [1, 2])
def test_reverberator_matches_oracle_across_blocks(ctx, sh_order):
    S = 2
    sc, p, prm, rev, cfg, pd = _setup(ctx, S, sh_order, 70 + sh_order)
    fs = 48000.0
    rng = np.random.default_rng(sh_order)
    N = 12192
    x = np.zeros((S, N), np.float32)
    x[:, 0] = 1.0
    x[:, 500:2500] += rng.normal(scale=0.3, size=(S, 2000)).astype(np.float32)
    R = rpr.Reverberator(ctx, S, sc.num_bands, p.K, XO, fs)
    xd = torch.tensor(x, device="cuda")
    cuts = ((0, 1), (1, 18), (18, 3000), (3000, 8000), (8000, 8033), (8033, N))
    parts = [R.render(rev, prm, xd[:, a:b]) for a, b in cuts]
    assert ctx.sync_status() == 0
    q = torch.cat(parts, dim=2).double().cpu().numpy()
    for s in range(S):
        qo = orv.render(x[s].astype(np.float64), cfg[s], pd["g_reverb"][s], pd["predelay_s"][s, 0], XO, fs)
        qo = qo.T  # [K][N]
        assert np.abs(qo).max() > 0
        rel = np.linalg.norm(q[s] - qo) / np.linalg.norm(qo)
        print(f"source {s}, SH order {sh_order}: relative L2 {rel:.2e}")
        assert rel < 1e-4, rel


def test_reverberator_batch_throughput(ctx):
    """256 sources, 4 bands, SH order 1 (the paper's reverberation order), 4096-sample
    blocks at 48 kHz: the device time of a block against its audio duration."""
    S, N = 256, 4096
    sc, p, prm, rev, cfg, pd = _setup(ctx, 1, 1, 75)
    rev_all = rev.repeat(S)
    prm_all = prm.repeat(S)
    R = rpr.Reverberator(ctx, S, sc.num_bands, p.K, XO, 48000.0)
    x = torch.randn((S, N), device="cuda") * 0.1
    for _ in range(2):
        R.render(rev_all, prm_all, x)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        R.render(rev_all, prm_all, x)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    audio_ms = 1000.0 * N / 48000.0
    print(f"reverberator: {S} sources x {N} samples in {ms:.3f} ms ({audio_ms / ms:.1f}x real time)")
    assert ctx.sync_status() == 0
    assert ms < audio_ms  # faster than real time
