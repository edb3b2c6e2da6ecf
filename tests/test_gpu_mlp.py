"""Learned estimator on the GPU: the BF16 tensor-core forward and backward kernels
against the FP64 oracle network (same BF16-rounded weights and inputs), AdamW against
the oracle's update, checkpoint/resume, and the gain of the trained network over the
plain estimator on low-ray-count IRs (both judged against high-ray labels)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1803_00430_gb300 import build, learned, rpr  # noqa: E402

DIN, DH, NH, DOUT = 528, 256, 3, 16


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = rpr.Context(0)
    yield c
    c.close()


def _bf16(x):
    return torch.as_tensor(x).float().bfloat16().double().numpy()


def _oracle_params(mlp, P):
    """The parameters the GPU kernels compute with: BF16 weights, FP32 biases."""
    P = P.double().cpu().numpy().copy()
    for W, b in oracle.mlp_split(P, DIN, DH, NH, DOUT):
        W[:] = _bf16(W)
    return P


def _setup(ctx, n=96, seed=0):
    mlp = rpr.MLP(ctx, max_batch=max(256, n), seed=seed + 11)
    rng = np.random.default_rng(seed)
    X = torch.tensor(rng.normal(size=(n, DIN)), dtype=torch.float32, device="cuda")
    Xb = mlp.prepare(X)  # identity normalisation
    T = torch.tensor(rng.normal(size=(n, DOUT)), dtype=torch.float32, device="cuda")
    M = torch.tensor((rng.uniform(size=(n, DOUT)) > 0.2).astype(np.float32), device="cuda")
    return mlp, X, Xb, T, M


def test_forward_matches_oracle(ctx):
    mlp, X, Xb, T, M = _setup(ctx)
    Yg = mlp.forward(Xb, destandardize=False).double().cpu().numpy()
    Po = _oracle_params(mlp, mlp.params())
    Yo = oracle.mlp_forward(Po, Xb.double().cpu().numpy(), DIN, DH, NH, DOUT)
    rel = np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo)
    assert rel < 1e-2, rel  # BF16 activations between layers


def test_gradients_match_oracle(ctx):
    mlp, X, Xb, T, M = _setup(ctx, seed=1)
    loss, g = mlp.loss_grad(Xb, T, M)
    g = g.double().cpu().numpy()
    Po = _oracle_params(mlp, mlp.params())
    lo, go = oracle.mlp_loss_grad(Po, Xb.double().cpu().numpy(), T.double().cpu().numpy(),
                                  M.double().cpu().numpy(), DIN, DH, NH, DOUT)
    assert float(loss.item()) == pytest.approx(lo, rel=2e-2)
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.999, cos
    for (Wg, bg), (Wo, bo) in zip(oracle.mlp_split(g, DIN, DH, NH, DOUT), oracle.mlp_split(go, DIN, DH, NH, DOUT)):
        assert np.linalg.norm(Wg - Wo) / np.linalg.norm(Wo) <= 2e-2
        assert np.linalg.norm(bg - bo) / np.linalg.norm(bo) <= 2e-2


def test_split_k_gradients_match_oracle(ctx):
    """1100 samples: the weight-gradient GEMMs split the batch dimension (5 ragged
    chunks) and the bias gradients sum it in row chunks."""
    mlp, X, Xb, T, M = _setup(ctx, n=1100, seed=5)
    loss, g = mlp.loss_grad(Xb, T, M)
    g = g.double().cpu().numpy()
    Po = _oracle_params(mlp, mlp.params())
    lo, go = oracle.mlp_loss_grad(Po, Xb.double().cpu().numpy(), T.double().cpu().numpy(),
                                  M.double().cpu().numpy(), DIN, DH, NH, DOUT)
    assert float(loss.item()) == pytest.approx(lo, rel=2e-2)
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.999, cos
    for (Wg, bg), (Wo, bo) in zip(oracle.mlp_split(g, DIN, DH, NH, DOUT), oracle.mlp_split(go, DIN, DH, NH, DOUT)):
        assert np.linalg.norm(Wg - Wo) / np.linalg.norm(Wo) <= 2e-2
        assert np.linalg.norm(bg - bo) / np.linalg.norm(bo) <= 2e-2
    # the same call twice gives the same bits (fixed reduction order)
    _, g2 = mlp.loss_grad(Xb, T, M)
    np.testing.assert_array_equal(g2.double().cpu().numpy(), g)


def test_adamw_step_matches_oracle(ctx):
    mlp, X, Xb, T, M = _setup(ctx, seed=2)
    P0 = mlp.params().double().cpu().numpy()
    _, g = mlp.loss_grad(Xb, T, M)
    g = g.double().cpu().numpy()
    lr, wd = 1e-3, 0.05
    mlp.train_step(Xb, T, M, lr, wd)
    P1 = mlp.params().double().cpu().numpy()
    Pe, m, v = P0.copy(), np.zeros_like(P0), np.zeros_like(P0)
    oracle.adamw_step(Pe, g, m, v, lr, 0.9, 0.999, 1e-8, wd, 1)
    np.testing.assert_allclose(P1, Pe, rtol=1e-5, atol=1e-7)


def test_checkpoint_resume_is_exact(ctx):
    mlp, X, Xb, T, M = _setup(ctx, seed=3)
    for _ in range(20):
        mlp.train_step(Xb, T, M, 1e-3, 1e-4)
    P, m, v, step = mlp.params(), *mlp.adam_state()
    for _ in range(10):
        mlp.train_step(Xb, T, M, 1e-3, 1e-4)
    Pa = mlp.params().cpu().numpy()
    other = rpr.MLP(ctx, max_batch=256, seed=999)
    other.set_params(P)
    other.set_adam_state(m, v, step)
    for _ in range(10):
        other.train_step(Xb, T, M, 1e-3, 1e-4)
    np.testing.assert_array_equal(other.params().cpu().numpy(), Pa)


def test_training_reduces_loss(ctx):
    mlp, X, Xb, T, M = _setup(ctx, n=256, seed=4)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    first = None
    for s in range(150):
        mlp.train_step(Xb, T, M, 3e-3, 0.0, loss)
        if s == 0:
            first = float(loss.item())
    assert float(loss.item()) < 0.2 * first  # 256 samples, 400k parameters: it memorises


def _gpu_features(ctx, H, sf, rate=1000.0, in_dim=528):
    Hd = torch.as_tensor(np.ascontiguousarray(H, np.float32), device="cuda")
    return rpr.mlp_features(ctx, Hd, sf, rate, in_dim).double().cpu().numpy()


def test_features_match_oracle_on_traced_irs(ctx):
    """Features of real IRs (a batched trace of procedural scenes) against the oracle."""
    scs = learned.learned_scenes(7, 24)
    rs = [rpr.Scene.from_scene(ctx, sc) for sc in scs]
    sf = np.stack([rpr.scene_features(s) for s in rs])
    p = rpr.TraceParams(**learned.TRACE)
    b = rpr.Batch(ctx, [(rs[i], scs[i].listener, scs[i].sources, 1500, i) for i in range(len(scs))], p)
    b.run(seed=99)
    H = b.H.double().cpu().numpy()
    Xg = rpr.mlp_features(ctx, b.H, sf, p.ir_rate_hz, 528).double().cpu().numpy()
    Xo = oracle.mlp_features(H, sf, p.ir_rate_hz, 528)
    # window lengths: equal unless the oracle's decay curve sits within rounding of
    # the -40 dB floor at the window's end
    tw_g, tw_o = Xg[:, 63:512:64], Xo[:, 63:512:64]
    same = np.abs(tw_g - tw_o) < 1e-6
    assert same.mean() >= 0.99, same.mean()
    for s, bnd in zip(*np.nonzero(~same)):
        t_o = int(round(np.exp(tw_o[s, bnd]) * p.ir_rate_hz))
        D = np.cumsum(H[s, bnd, 0, ::-1])[::-1] / H[s, bnd, 0].sum()
        assert abs(D[t_o - 1] / 1e-4 - 1) < 1e-5 or abs(D[t_o] / 1e-4 - 1) < 1e-5
    cols = np.concatenate([np.arange(b * 64, b * 64 + 63) for b in range(8)])
    rows_ok = np.repeat(same, 63, axis=1)
    np.testing.assert_allclose(Xg[:, cols][rows_ok], Xo[:, cols][rows_ok], rtol=0, atol=2e-5)
    np.testing.assert_allclose(Xg[:, 512:], Xo[:, 512:], rtol=1e-6, atol=1e-6)
    b.close()


def test_features_edge_cases(ctx):
    rng = np.random.default_rng(8)
    sf = rng.normal(size=(3, 10))
    # 3 bands, 4 SH coefficients, an impulse, an empty band, a short IR at 4 bins
    for T in (4, 5, 257, 3000):
        H = np.zeros((3, 3, 4, T))
        H[0, 0, 0, min(2, T - 1)] = 1.0
        H[1, 1, 0] = np.exp(-np.arange(T) / 50.0)
        H[:, :, 1:] = rng.normal(size=(3, 3, 3, T))
        H[2, 2, 0] = rng.uniform(size=T) * np.exp(-np.arange(T) / 9.0)
        Xg = _gpu_features(ctx, H, sf, 2000.0, 536)
        Xo = oracle.mlp_features(H.astype(np.float32).astype(np.float64), sf.astype(np.float32), 2000.0, 536)
        np.testing.assert_allclose(Xg, Xo, rtol=0, atol=2e-5)
    with pytest.raises(rpr.RprError):
        _gpu_features(ctx, np.zeros((1, 1, 1, 11265)), sf[:1])
    with pytest.raises(rpr.RprError):
        _gpu_features(ctx, np.zeros((1, 1, 1, 3)), sf[:1])


def test_learned_estimator_gains_over_plain(ctx):
    """Trained on the method's own IRs (2k-ray inputs, labels from 100k-ray traces),
    the network's decay times beat the plain estimator's on the same held-out 2k-ray
    IRs, in the mean and in the 95th percentile of the relative error."""
    train = learned.make_dataset(ctx, 2048, seed=101, low_rays=(2000,), high_rays=100000, copies=4)
    test = learned.make_dataset(ctx, 256, seed=202, low_rays=(2000,), high_rays=200000)
    mlp, hist = learned.fit(ctx, train, steps=3000, batch=512, lr=1e-3, weight_decay=1e-2, log_every=1000)
    ev = learned.evaluate(mlp, test)
    print("learned vs plain (held out):", ev, "loss", hist, "labels", train.label_frac, test.label_frac)
    assert ev["n"] > 1000
    assert hist[-1][1] < 0.5 * hist[0][1]
    assert ev["rt_err_mean_net"] < ev["rt_err_mean_plain"]
    assert ev["rt_err_p95_net"] < ev["rt_err_p95_plain"]


@pytest.mark.parametrize("n", [1, 100, 128, 300, 4097])
def test_tensor_core_forward_matches_gemm_forward_and_oracle(ctx, n):
    """The fused tcgen05 forward pass (TMA-staged operands, TMEM accumulators, one
    launch for all layers) against the mma.sync GEMM path on the same weights and
    inputs, and against the FP64 oracle; ragged batches (1, a partial 128-sample tile,
    a tile and a tail) and the 528-wide input's partial last K-chunk."""
    rng = np.random.default_rng(100 + n)
    tc = rpr.MLP(ctx, max_batch=max(n, 256), seed=21)
    ref = rpr.MLP(ctx, max_batch=max(n, 256), seed=22, legacy_gemm=True)
    ref.set_params(tc.params())
    X = torch.tensor(rng.normal(size=(n, DIN)), dtype=torch.float32, device="cuda")
    Xb = tc.prepare(X)
    Yt = tc.forward(Xb, destandardize=False).double().cpu().numpy()
    Yr = ref.forward(Xb, destandardize=False).double().cpu().numpy()
    assert np.isfinite(Yt).all()
    rel = np.linalg.norm(Yt - Yr) / np.linalg.norm(Yr)
    # same BF16 activations up to FP32 accumulation order (a rounding flip of a BF16
    # activation moves the output by about 2^-9 of one term)
    assert rel < 2e-3, rel
    Po = _oracle_params(tc, tc.params())
    Yo = oracle.mlp_forward(Po, Xb.double().cpu().numpy(), DIN, DH, NH, DOUT)
    assert np.linalg.norm(Yt - Yo) / np.linalg.norm(Yo) < 1e-2
    assert ctx.sync_status() == 0


def test_tensor_core_forward_keeps_training_state(ctx):
    """Training runs the tcgen05 forward pass with the pre-activations and BF16
    activations kept for the backward pass: gradients equal the GEMM path's."""
    n = 700
    rng = np.random.default_rng(7)
    tc = rpr.MLP(ctx, max_batch=n, seed=31)
    ref = rpr.MLP(ctx, max_batch=n, seed=32, legacy_gemm=True)
    ref.set_params(tc.params())
    X = torch.tensor(rng.normal(size=(n, DIN)), dtype=torch.float32, device="cuda")
    Xb = tc.prepare(X)
    T = torch.tensor(rng.normal(size=(n, DOUT)), dtype=torch.float32, device="cuda")
    M = torch.ones((n, DOUT), dtype=torch.float32, device="cuda")
    lt, gt = tc.loss_grad(Xb, T, M)
    lr, gr = ref.loss_grad(Xb, T, M)
    gt, gr = gt.double().cpu().numpy(), gr.double().cpu().numpy()
    assert float(lt.item()) == pytest.approx(float(lr.item()), rel=1e-3)
    cos = float(gt @ gr / (np.linalg.norm(gt) * np.linalg.norm(gr)))
    assert cos >= 0.9999, cos
    assert np.linalg.norm(gt - gr) / np.linalg.norm(gr) < 1e-2
