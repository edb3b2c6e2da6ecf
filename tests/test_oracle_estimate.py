"""Pins of the oracle's reverberation-parameter estimator (paper Section 4.2).

* A pure exponential IR I_j = r^j with r = 10^(-6 / (RT f)) must give RT60 = RT to
  1e-9 and g_reverb = sqrt(sum r^j / (RT / (6 ln 10))) (the paper's closed form
  I_reverb^total = RT60 / (6 ln 10)).
* An IR too short to reach the T30 floor must fall back to T20; the fit is checked
  against numpy.polyfit of the closed-form Schroeder curve of a flat IR.
* Empty IRs give no decay time; predelay, DRR, directivity and smoothing are checked
  against their definitions on synthetic inputs with known answers.
"""
import numpy as np
import pytest


def _H_from_I(I, K=4, direction=None, order=1):
    """Histogram with intensity I in band 0 (H_00 = I / sqrt(4 pi))."""
    S, B, T = I.shape
    H = np.zeros((S, B, K, T))
    H[:, :, 0, :] = I / np.sqrt(4 * np.pi)
    return H


@pytest.mark.parametrize("rt,f", [(0.5, 1000.0), (1.7, 1000.0), (2.5, 100.0)])
def test_pure_exponential_decay(oracle_lib, rt, f):
    T = int(np.ceil(3 * rt * f))
    r = 10 ** (-6 / (rt * f))
    I = (r ** np.arange(T))[None, None, :] * 0.01
    ep = oracle_lib.estimate(_H_from_I(I), np.array([0.0]), f)
    assert ep["range_kind"][0, 0] == 1
    assert ep["rt60_raw"][0, 0] == pytest.approx(rt, rel=1e-9)
    itot = 0.01 * (1 - r ** T) / (1 - r)
    assert ep["i_total"][0, 0] == pytest.approx(itot, rel=1e-12)
    assert ep["g_reverb"][0, 0] == pytest.approx(np.sqrt(itot / (rt / (6 * np.log(10)))), rel=1e-9)
    # comb gain of Eq. (comb_feedback_gain) with t_comb = 1 reproduces the decay:
    # 20 log10 g^RT = -60 dB
    g = 10 ** (-3 * 1.0 / ep["rt60_raw"][0, 0])
    assert 20 * np.log10(g ** rt) == pytest.approx(-60, rel=1e-9)
    assert ep["fit_r2"][0, 0] == pytest.approx(1.0, abs=1e-12)


def test_short_ir_falls_back_to_t20(oracle_lib):
    f = 1000.0
    T = 450
    # flat IR: the Schroeder curve is 10 log10((T - j) / T) and ends at
    # 10 log10(1/450) = -26.5 dB, so the T30 floor (-35 dB) is never reached
    j = np.arange(T)
    I = np.full((1, 1, T), 0.02)
    ep = oracle_lib.estimate(_H_from_I(I), np.array([0.0]), f)
    assert ep["range_kind"][0, 0] == 2
    Ld = 10 * np.log10((T - j) / T)
    sel = (Ld <= -5) & (Ld >= -25)
    slope = np.polyfit(j[sel] / f, Ld[sel], 1)[0]
    assert ep["rt60_raw"][0, 0] == pytest.approx(-60 / slope, rel=1e-9)
    assert ep["n_fit"][0, 0] == sel.sum()
    assert ep["fit_j0"][0, 0] == np.nonzero(sel)[0][0] and ep["fit_j1"][0, 0] == np.nonzero(sel)[0][-1]


def test_t10_fallback_and_none(oracle_lib):
    f = 1000.0
    T = 60
    r = 10 ** (-6 / (1.0 * f))
    I = np.zeros((1, 3, T))
    I[0, 0] = r ** np.arange(T)
    I[0, 1, :5] = 1.0                    # five equal bins: Schroeder curve 0, -1, -2.2, -4, -7 dB
    ep = oracle_lib.estimate(_H_from_I(I), np.zeros(1), f)
    assert ep["range_kind"][0, 1] == 3   # T10 from 0..-10 dB
    assert ep["range_kind"][0, 2] == 0 and np.isnan(ep["rt60_raw"][0, 2])
    assert np.isnan(ep["g_reverb"][0, 2])
    # predelay is per source, the first bin that is non-zero in any band
    assert ep["predelay_s"][0, 2] == 0.0


def test_predelay_drr_and_directivity(oracle_lib):
    f = 100.0
    S, B, K, T = 2, 3, 4, 50
    H = np.zeros((S, B, K, T))
    rng = np.random.default_rng(0)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    Y = oracle_lib.sh_eval(1, d)
    # source 0: first energy at bin 7 in band 2 only, later bins in all bands
    H[0, 2, :, 7] = 0.3 * Y
    H[0, :, :, 9:20] = 0.1 * Y[None, :, None]
    # source 1: nothing
    ed = np.array([0.05, 0.0])
    ep = oracle_lib.estimate(H, ed, f)
    assert ep["predelay_s"][0, 0] == pytest.approx(7 / f)
    assert ep["predelay_s"][0, 1] == pytest.approx(7 / f)
    assert np.isnan(ep["predelay_s"][1, 0])
    itot = 1.1 * 1.0  # 11 bins of energy 0.1 (I = sqrt(4pi) * 0.1 * Y00 = 0.1)
    assert ep["i_total"][0, 0] == pytest.approx(itot, rel=1e-12)
    assert ep["drr_db"][0, 0] == pytest.approx(10 * np.log10(0.05 / itot), rel=1e-12)
    # all contributions from one direction: X-bar equals Y(d)
    np.testing.assert_allclose(ep["xbar"][0, 1], Y, rtol=1e-12)
    x = ep["xbar"][0, 2]
    xm = np.array([-x[3], -x[1], x[2]])
    np.testing.assert_allclose(xm / np.linalg.norm(xm), d, atol=1e-12)
    assert np.isnan(ep["drr_db"][1, 0])


def test_exponential_smoothing(oracle_lib):
    rt, f = 1.2, 1000.0
    T = 4000
    r = 10 ** (-6 / (rt * f))
    I = (r ** np.arange(T))[None, None, :]
    H = _H_from_I(I)
    state = np.full((1, 1), np.nan)
    ep = oracle_lib.estimate(H, np.zeros(1), f, dt_update=0.1, tau=3.0, state=state)
    assert ep["rt60_smoothed"][0, 0] == pytest.approx(rt, rel=1e-9)  # first update takes the value
    for _ in range(5):  # constant input: fixed point
        ep = oracle_lib.estimate(H, np.zeros(1), f, dt_update=0.1, tau=3.0, state=state)
    assert state[0, 0] == pytest.approx(rt, rel=1e-9)
    # step to a new decay time: after tau seconds of updates the remaining gap is 1/e
    rt2 = 0.6
    r2 = 10 ** (-6 / (rt2 * f))
    H2 = _H_from_I((r2 ** np.arange(T))[None, None, :])
    dt, tau = 0.05, 3.0
    for _ in range(int(round(tau / dt))):
        ep = oracle_lib.estimate(H2, np.zeros(1), f, dt_update=dt, tau=tau, state=state)
    gap = (state[0, 0] - rt2) / (rt - rt2)
    assert gap == pytest.approx(np.exp(-1.0), rel=1e-9)
