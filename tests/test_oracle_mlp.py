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
