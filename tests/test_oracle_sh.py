"""Pins of the oracle's real spherical harmonics (paper Section 2 "Spherical
Harmonics", Section 4.1 dominant-direction formula).

Checked against scipy's complex spherical harmonics (a library routine) converted
to the real basis, against closed forms on the coordinate axes, by quadrature
orthonormality, and by the paper's first-order dominant-direction formula
x_max = normalize(-X_{1,1}, -X_{1,-1}, X_{1,0}), which fixes the sign convention.
"""
import numpy as np
import pytest
from scipy import special


def _real_sh_scipy(order, d):
    d = np.asarray(d, float) / np.linalg.norm(d)
    theta = np.arccos(np.clip(d[2], -1, 1))
    phi = np.arctan2(d[1], d[0])
    out = np.zeros((order + 1) ** 2)
    for l in range(order + 1):
        for m in range(-l, l + 1):
            y = special.sph_harm_y(l, abs(m), theta, phi)  # includes Condon-Shortley
            if m > 0:
                v = np.sqrt(2) * y.real
            elif m < 0:
                v = np.sqrt(2) * y.imag
            else:
                v = y.real
            out[l * l + l + m] = v
    return out


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4])
def test_sh_matches_scipy(oracle_lib, order):
    rng = np.random.default_rng(order)
    for _ in range(200):
        d = rng.normal(size=3)
        np.testing.assert_allclose(oracle_lib.sh_eval(order, d), _real_sh_scipy(order, d),
                                   rtol=1e-12, atol=1e-13)


def test_sh_closed_forms_on_axes(oracle_lib):
    c0 = 1 / (2 * np.sqrt(np.pi))
    c1 = np.sqrt(3 / (4 * np.pi))
    c20 = np.sqrt(5 / (16 * np.pi))
    for d, y1 in [((1, 0, 0), (0, 0, -c1)), ((-1, 0, 0), (0, 0, c1)), ((0, 1, 0), (-c1, 0, 0)),
                  ((0, -1, 0), (c1, 0, 0)), ((0, 0, 1), (0, c1, 0)), ((0, 0, -1), (0, -c1, 0))]:
        Y = oracle_lib.sh_eval(2, d)
        assert Y[0] == pytest.approx(c0, abs=1e-15)
        np.testing.assert_allclose(Y[1:4], y1, atol=1e-15)
        # Y_20 = sqrt(5/16pi) (3 z^2 - 1)
        assert Y[6] == pytest.approx(c20 * (3 * d[2] ** 2 - 1), abs=1e-14)


def test_sh_orthonormal_by_quadrature(oracle_lib):
    order = 3
    K = (order + 1) ** 2
    xg, wg = np.polynomial.legendre.leggauss(24)  # exact in cos(theta) for these degrees
    nphi = 48
    G = np.zeros((K, K))
    for z, w in zip(xg, wg):
        r = np.sqrt(1 - z * z)
        for j in range(nphi):
            ph = 2 * np.pi * j / nphi
            Y = oracle_lib.sh_eval(order, (r * np.cos(ph), r * np.sin(ph), z))
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(K), atol=1e-10)


def test_dominant_direction_recovers_single_direction(oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        X = 0.37 * oracle_lib.sh_eval(1, d)  # one contribution of energy 0.37
        xmax = np.array([-X[3], -X[1], X[2]])
        np.testing.assert_allclose(xmax / np.linalg.norm(xmax), d, atol=1e-12)
