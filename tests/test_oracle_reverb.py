"""Pins of the oracle's reverberator parameters (Sections 4.1 and 4.2).

  * The sphere rule integrates products of SH exactly (orthonormality).
  * SH rotations: Y(R d) = J(R) Y(d) for random directions, J orthogonal and block
    diagonal by degree, J(R1 R2) = J(R1) J(R2).
  * Directional loudness: the identity for isotropic reverberation; its trace follows
    the SH addition theorem, sum_k Y_k(x)^2 = (n + 1)^2 / (4 pi).
  * Comb gains: a comb of delay t and gain g decays by 60 dB in RT60 (g^(RT60/t) = 1e-3).
  * Comb delays: Gaussian about r_free / c with sigma = mean / 3 (moments within
    their sampling error), redrawn only when the mean moves by more than 2 sigma.
  * Comb input direction: the direction of a single-direction IR, and the linear
    interpolation between two bins.
  * Comb rotations: angles in [90, 270] degrees, R orthonormal with det 1.
"""
import numpy as np
import pytest

import oracle
from oracle import reverb


@pytest.mark.parametrize("order", [1, 2, 3])
def test_sphere_rule_integrates_sh_products_exactly(order):
    dirs, w = reverb.sphere_rule(order)
    Y = reverb.sh_matrix(order, dirs)
    np.testing.assert_allclose((Y * w[:, None]).T @ Y, np.eye((order + 1) ** 2), atol=1e-13)
    assert w.sum() == pytest.approx(4 * np.pi, rel=1e-14)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_sh_rotation_rotates_directions(order):
    rng = np.random.default_rng(order)
    R1, _ = reverb.comb_rotation(7, 0, 1)
    R2, _ = reverb.comb_rotation(7, 3, 5)
    J1, J2 = reverb.sh_rotation(R1, order), reverb.sh_rotation(R2, order)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        np.testing.assert_allclose(oracle.sh_eval(order, R1 @ d), J1 @ oracle.sh_eval(order, d), atol=1e-12)
    np.testing.assert_allclose(J1 @ J1.T, np.eye(J1.shape[0]), atol=1e-12)
    np.testing.assert_allclose(reverb.sh_rotation(R1 @ R2, order), J1 @ J2, atol=1e-12)
    for l in range(order + 1):  # no mixing between degrees
        lo, hi = l * l, (l + 1) ** 2
        off = J1[lo:hi].copy()
        off[:, lo:hi] = 0.0
        assert np.abs(off).max() < 1e-12


def test_directional_loudness_identity_and_trace():
    for order in (1, 2, 3):
        K = (order + 1) ** 2
        iso = np.zeros(K)
        iso[0] = 0.7
        np.testing.assert_allclose(reverb.directional_loudness(iso, order), np.eye(K), atol=1e-12)
        d = np.array([0.3, -0.5, 0.81])
        d /= np.linalg.norm(d)
        xbar = 0.5 * oracle.sh_eval(order, d) / oracle.sh_eval(order, d)[0] * 0.28209479177387814
        D = reverb.directional_loudness(xbar, order)
        np.testing.assert_allclose(D, D.T, atol=1e-14)
        dirs, w = reverb.sphere_rule(order)
        f = reverb.sh_matrix(order, dirs) @ xbar
        a = np.sqrt(np.maximum(f, 0) / (xbar[0] * 0.28209479177387814))
        assert np.trace(D) == pytest.approx(K / (4 * np.pi) * (w * a).sum(), rel=1e-12)
        # louder towards d than away from it
        y = oracle.sh_eval(order, d)
        assert y @ D @ y > (-y) @ D @ (-y) * 0.999 and np.linalg.norm(D @ y) > np.linalg.norm(D @ oracle.sh_eval(order, -d))


def test_comb_delays_moments_and_redraw_rule():
    mean = 0.0123
    t = np.concatenate([reverb.draw_delays(11, s, g, mean) for s in range(25) for g in range(1, 21)])
    n = len(t)
    sigma = mean / 3
    assert abs(t.mean() - mean) < 4 * sigma / np.sqrt(n)
    assert abs(t.std() - sigma) < 0.08 * sigma
    assert t.min() >= mean / 10
    # redraw when r_free / c moves by more than 2 sigma (of the mean the delays were drawn for)
    H = np.zeros((1, 1, 1, 10))
    H[0, 0, 0, 2] = 1.0
    rt, xb, st, gens = np.array([[1.0]]), np.zeros((1, 1, 1)), None, []
    for mfp in [3.43, 3.43 * 1.5, 3.43 * 1.7, 3.43 * 1.71, 3.43 * 1.0]:
        out, st = reverb.configure(H, rt, xb, mfp, 343.0, 100.0, 5, st)
        gens.append(out[0]["generation"])
    # 1.5: moved 0.5 mean < 2/3 mean: kept; 1.7: moved 0.7 > 2/3: redrawn (new mean 1.7);
    # 1.71: kept; back to 1.0: moved 0.7 of 1.7 < 2/3 x 1.7: kept
    assert gens == [1, 1, 2, 2, 2]


def test_comb_gains_decay_60_db_in_rt60():
    H = np.zeros((1, 2, 4, 50))
    H[0, :, 0, 3] = 1.0
    rt = np.array([[0.8, 2.5]])
    out, _ = reverb.configure(H, rt, np.zeros((1, 2, 4)), 5.0, 343.0, 100.0, 9, None)
    t, g = out[0]["t_comb"], out[0]["g_comb"]
    for i in range(reverb.N_COMB):
        for b in range(2):
            assert g[i][b] ** (rt[0][b] / t[i]) == pytest.approx(1e-3, rel=1e-12)


def test_comb_direction_of_a_single_direction_ir_and_interpolation():
    order, T = 2, 40
    d1 = np.array([0.2, 0.9, -0.3]); d1 /= np.linalg.norm(d1)
    d2 = np.array([-0.7, 0.1, 0.5]); d2 /= np.linalg.norm(d2)
    H = np.zeros((3, 9, T))
    for j in range(5, T):
        H[:, :, j] = 0.2 * oracle.sh_eval(order, d1)[None, :]
    np.testing.assert_allclose(reverb.comb_direction(H, 0.0731, 100.0), d1, atol=1e-12)
    H[:, :, 12] = 0.2 * oracle.sh_eval(order, d2)[None, :]
    x = 5 + 0.0731 * 100.0 - 0.0  # bin 12.31: between bins 12 (d2) and 13 (d1)
    f = x - 12
    v = (1 - f) * d2 + f * d1
    np.testing.assert_allclose(reverb.comb_direction(H, 0.0731, 100.0), v / np.linalg.norm(v), atol=1e-12)


def test_comb_rotations_span_90_to_270_degrees():
    for s in range(5):
        for i in range(reverb.N_COMB):
            R, a = reverb.comb_rotation(123, s, i)
            assert ((a >= np.pi / 2) & (a < 1.5 * np.pi)).all()
            np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
            assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
