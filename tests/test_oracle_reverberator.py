"""Pins of the oracle's SH-domain Schroeder reverberator (Section 4.1):

  * a Linkwitz-Riley crossover's low and high parts add up to an all-pass (unit
    magnitude at every frequency), each -6 dB at the crossover frequency;
  * a comb filter's impulse response is g^k J^k at k delays (closed form);
  * an all-pass filter keeps the energy of an impulse;
  * the whole reverberator, with comb gains 10^(-3 t_comb / RT60), decays by 60 dB
    in RT60 (its output's Schroeder decay fitted between -5 and -35 dB).
"""
import numpy as np
import pytest

scipy_signal = pytest.importorskip("scipy.signal")

from oracle import reverb, reverberator as rv  # noqa: E402


def test_lr4_crossover_sums_to_an_allpass_and_is_minus_6_db_at_fc():
    fs = 48000.0
    for fc in (176.0, 775.0, 3408.0):
        x = np.zeros(1 << 16)
        x[0] = 1.0
        s = rv.lr4(x, fc, fs, False) + rv.lr4(x, fc, fs, True)
        np.testing.assert_allclose(np.abs(np.fft.rfft(s)), 1.0, atol=1e-6)
        for high in (False, True):
            b, a = rv.butterworth2(fc, fs, high)
            _, h = scipy_signal.freqz(b, a, worN=[2 * np.pi * fc / fs])
            assert abs(h[0]) ** 2 == pytest.approx(0.5, rel=1e-9)  # LR4 = the biquad squared: -6 dB


def test_comb_impulse_response_is_gain_and_rotation_powers():
    R, _ = reverb.comb_rotation(3, 0, 2)
    J = reverb.sh_rotation(R, 1)
    u = np.zeros((400, 4))
    u0 = np.array([0.3, -0.2, 0.5, 0.1])
    u[0] = u0
    y = rv.comb(u, 0.8, J, 37)
    for k in range(0, 400 // 37 + 1):
        np.testing.assert_allclose(y[37 * k], 0.8 ** k * np.linalg.matrix_power(J, k) @ u0, atol=1e-13)
    mask = np.ones(400, bool)
    mask[::37] = False
    assert np.abs(y[mask]).max() == 0.0


def test_allpass_keeps_the_energy_of_an_impulse():
    u = np.zeros((200000, 1))
    u[0] = 1.0
    for d in (1, 29, 240):
        v = rv.allpass(u, rv.AP_GAIN, d)
        assert (v ** 2).sum() == pytest.approx(1.0, abs=1e-9)


def test_reverberator_decays_60_db_in_rt60():
    fs, rt = 48000.0, 0.6
    H = np.zeros((1, 1, 4, 10))
    H[0, 0, 0, 1] = 1.0
    out, _ = reverb.configure(H, np.array([[rt]]), np.array([[[0.2821, 0, 0, 0]]]), 8.0, 343.0, 100.0, 17, None)
    r = out[0]
    x = np.zeros(int(1.2 * rt * fs))
    x[0] = 1.0
    q = rv.render(x, r, [1.0], 0.0, [], fs)
    e = (q ** 2).sum(axis=1)
    edc = np.cumsum(e[::-1])[::-1]
    L = 10 * np.log10(edc / edc[0])
    sel = (L <= -5) & (L >= -35)
    t = np.arange(len(L)) / fs
    slope = np.polyfit(t[sel], L[sel], 1)[0]
    assert -60.0 / slope == pytest.approx(rt, rel=0.05)
