"""Pins of the oracle's learned-estimator network (oracle/mlp.c): affine layers
against numpy's matmul, GELU against x * Phi(x) from scipy's normal CDF, the
gradient against central finite differences, the masked loss definition, and
AdamW against torch.optim.AdamW and its first-step closed form."""
import numpy as np
import pytest
from scipy import stats


def _rand_params(o, rng, din, dh, nh, dout, scale=0.5):
    return rng.normal(scale=scale, size=o.mlp_param_count(din, dh, nh, dout))


def test_affine_network_is_a_matmul(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(0)
    din, dout = 7, 5
    P = _rand_params(o, rng, din, 3, 0, dout)
    X = rng.normal(size=(11, din))
    (W, b), = o.mlp_split(P, din, 3, 0, dout)
    np.testing.assert_allclose(o.mlp_forward(P, X, din, 3, 0, dout), X @ W + b, rtol=1e-13, atol=1e-13)


def test_gelu_layer(oracle_lib):
    o = oracle_lib
    d = 6
    P = np.zeros(o.mlp_param_count(d, d, 1, d))
    (W1, b1), (W2, b2) = o.mlp_split(P, d, d, 1, d)
    W1[:] = np.eye(d)
    W2[:] = np.eye(d)
    X = np.linspace(-4, 4, 5 * d).reshape(5, d)
    np.testing.assert_allclose(o.mlp_forward(P, X, d, d, 1, d), X * stats.norm.cdf(X), rtol=1e-13, atol=1e-15)


def test_gradient_matches_finite_differences(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(1)
    din, dh, nh, dout, n = 9, 6, 3, 4, 7
    P = _rand_params(o, rng, din, dh, nh, dout)
    X = rng.normal(size=(n, din))
    T = rng.normal(size=(n, dout))
    M = (rng.uniform(size=(n, dout)) > 0.3).astype(float)
    loss, G = o.mlp_loss_grad(P, X, T, M, din, dh, nh, dout)
    h = 1e-6
    idx = rng.choice(P.size, size=60, replace=False)
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (o.mlp_loss_grad(Pp, X, T, M, din, dh, nh, dout)[0] - o.mlp_loss_grad(Pm, X, T, M, din, dh, nh, dout)[0]) / (2 * h)
        assert G[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_masked_loss_definition(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(2)
    din, dh, nh, dout, n = 5, 4, 2, 3, 6
    P = _rand_params(o, rng, din, dh, nh, dout)
    X = rng.normal(size=(n, din))
    Y = o.mlp_forward(P, X, din, dh, nh, dout)
    M = np.ones((n, dout))
    M[2, 1] = 0.0
    T = Y.copy()
    assert o.mlp_loss_grad(P, X, T, M, din, dh, nh, dout)[0] == 0.0
    T[2, 1] += 10.0  # a masked entry does not count
    assert o.mlp_loss_grad(P, X, T, M, din, dh, nh, dout)[0] == 0.0
    T[0, 0] += 3.0
    assert o.mlp_loss_grad(P, X, T, M, din, dh, nh, dout)[0] == pytest.approx(9.0 / M.sum(), rel=1e-12)


def test_adamw_matches_torch_and_first_step(oracle_lib):
    o = oracle_lib
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=lr, betas=(b1, b2), eps=eps, weight_decay=wd)
    for step in range(1, 6):
        g = rng.normal(size=50)
        if step == 1:
            # closed form of the first step: m_hat = g, v_hat = g^2
            expect = p - lr * (g / (np.abs(g) + eps) + wd * p)
        o.adamw_step(p, g, m, v, lr, b1, b2, eps, wd, step)
        if step == 1:
            np.testing.assert_allclose(p, expect, rtol=1e-12)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-10, atol=1e-14)


def _features(o, H, rate=1000.0, scene=None, in_dim=528):
    S = H.shape[0]
    if scene is None:
        scene = np.arange(S * 10, dtype=np.float64).reshape(S, 10) * 0.1
    return o.mlp_features(H, scene, rate, in_dim)


def test_features_of_a_geometric_decay(oracle_lib):
    """h(t) = q^t: D(t)/D(0) = (q^t - q^T) / (1 - q^T) (finite geometric series)."""
    o = oracle_lib
    T, rate = 1500, 1000.0
    q = 10 ** (-60.0 / 10.0 / (0.8 * rate))  # RT60 0.8 s
    H = np.zeros((1, 2, 4, T))
    H[0, 1, 0] = q ** np.arange(T)
    H[0, 1, 1:] = np.random.default_rng(3).normal(size=(3, T))  # k > 0 is not read
    X = _features(o, H, rate)[0]

    def r(t):
        return (q ** t - q ** T) / (1 - q ** T)

    first = int(np.argmax(r(np.arange(T)) < 1e-4))
    assert 0.8 * 40 / 60 * rate - 2 <= first <= 0.8 * 40 / 60 * rate + 2
    assert X[64 + 63] == pytest.approx(np.log(first / rate), rel=1e-12)
    for i in range(63):
        pos = first * (i + 1) / 63
        i0 = int(np.floor(pos))
        w = pos - i0
        assert X[64 + i] == pytest.approx(np.log10(r(i0) * (1 - w) + r(i0 + 1) * w + 1e-8), abs=1e-10)
    # band 0 is empty: -8 and the shortest window
    np.testing.assert_allclose(X[:63], -8.0, atol=1e-12)
    assert X[63] == pytest.approx(np.log(4 / rate))


def test_features_of_an_impulse_and_the_window_clamps(oracle_lib):
    o = oracle_lib
    T, k = 200, 37
    H = np.zeros((1, 1, 1, T))
    H[0, 0, 0, k] = 2.5
    X = _features(o, H)[0]
    assert X[63] == pytest.approx(np.log((k + 1) / 1000.0))
    for i in range(63):
        pos = (k + 1) * (i + 1) / 63
        expect = 1.0 if pos <= k else 1.0 - (pos - k)
        assert X[i] == pytest.approx(np.log10(expect + 1e-8), abs=1e-12)
    # a 4-bin IR with an impulse in bin 0: window of 4 bins, positions clamped to 2.999
    H4 = np.zeros((1, 1, 1, 4))
    H4[0, 0, 0, 0] = 1.0
    X4 = _features(o, H4)[0]
    assert X4[63] == pytest.approx(np.log(4 / 1000.0))
    assert X4[62] == pytest.approx(-8.0, abs=1e-9)  # clamped into the last bins, which are empty
    assert X4[0] == pytest.approx(np.log10(1 - 4 / 63 + 1e-8), abs=1e-12)
    # bands beyond B are empty bands
    np.testing.assert_allclose(X4[64:64 * 8].reshape(7, 64)[:, :63], -8.0, atol=1e-12)


def test_features_are_scale_free_and_place_the_scene_features(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(5)
    T = 400
    H = np.exp(-np.arange(T) / rng.uniform(20, 80, size=(3, 8, 1, 1))) * rng.uniform(0.5, 2, size=(3, 8, 1, T))
    sc = rng.normal(size=(3, 10))
    X1 = o.mlp_features(H, sc, 1000.0, 536)
    X2 = o.mlp_features(H * 7.3, sc, 1000.0, 536)
    np.testing.assert_allclose(X1, X2, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(X1[:, 512:522], sc)
    np.testing.assert_array_equal(X1[:, 522:], 0.0)
    # the same IR at twice the rate is the same decay curve over half the time
    X3 = o.mlp_features(H, sc, 2000.0, 536)
    np.testing.assert_allclose(X3[:, 63:512:64], X1[:, 63:512:64] - np.log(2.0), atol=1e-12)
