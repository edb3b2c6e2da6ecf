"""FP64 oracle of the SH-domain Schroeder reverberator (Section 4.1 "Sound Rendering";
Section 5 "Auralization"), test infrastructure only.  For each source, from its mono
input s(t):

  1. bands: a serial Linkwitz-Riley 4th-order crossover -- band 0 is the low-pass at
     the first crossover frequency, the high-pass part is split again at the next, and
     so on; band B-1 is the last high-pass part.  An LR4 section is a 2nd-order
     Butterworth biquad (bilinear transform with the crossover frequency prewarped)
     applied twice;
  2. the reverberator input reads each band at the predelay (round(t_predelay fs)
     samples, 0 when undefined);
  3. N_comb comb filters in parallel in the SH domain: comb i of band b holds a
     K-vector, y[n] = comb_in_i x_b[n - p] + g_comb[i][b] J_i y[n - d_i],
     d_i = max(1, round(t_comb_i fs)) -- each pass through the feedback multiplies the
     delayed vector by the comb's SH rotation J_i and its gain;
  4. the combs' sum through N_ap = 4 all-pass filters in series per channel,
     v[n] = -a u[n] + u[n - d] + a v[n - d], a = 0.7, d = 5, 1.7, 0.6 and 0.2 ms
     [reading: the paper gives only the counts];
  5. output q[n] = sum_b g_reverb[b] D_b v_b[n] (K SH channels).

scipy.signal.lfilter serves as the biquad step; the rest is plain numpy.
"""
from __future__ import annotations

import numpy as np

AP_GAIN = 0.7
AP_DELAYS_MS = (5.0, 1.7, 0.6, 0.2)


def butterworth2(fc: float, fs: float, high: bool):
    """2nd-order Butterworth low- or high-pass biquad (b, a) by the bilinear transform."""
    k = np.tan(np.pi * fc / fs)
    q = np.sqrt(2.0)
    norm = 1.0 / (1.0 + q * k + k * k)
    a = np.array([1.0, 2.0 * (k * k - 1.0) * norm, (1.0 - q * k + k * k) * norm])
    if high:
        b = np.array([norm, -2.0 * norm, norm])
    else:
        b0 = k * k * norm
        b = np.array([b0, 2.0 * b0, b0])
    return b, a


def lr4(x, fc: float, fs: float, high: bool):
    from scipy.signal import lfilter
    b, a = butterworth2(fc, fs, high)
    return lfilter(b, a, lfilter(b, a, x))


def split_bands(x, crossovers, fs: float):
    bands, rest = [], np.asarray(x, float)
    for fc in crossovers:
        bands.append(lr4(rest, fc, fs, False))
        rest = lr4(rest, fc, fs, True)
    bands.append(rest)
    return bands


def delay_samples(t: float, fs: float) -> int:
    return 0 if not np.isfinite(t) else max(0, int(np.floor(t * fs + 0.5)))


def comb(u, g: float, J, d: int):
    """y[n] = u[n] + g J y[n - d] for a [N][K] input, chunks of d samples at a time."""
    y = np.array(u, float, copy=True)
    N = len(y)
    for c in range(d, N, d):
        e = min(c + d, N)
        y[c:e] += g * (y[c - d:e - d] @ np.asarray(J).T)
    return y


def allpass(u, a: float, d: int):
    """v[n] = -a u[n] + u[n - d] + a v[n - d] along axis 0."""
    u = np.asarray(u, float)
    v = -a * u
    v[d:] += u[:-d] if d > 0 else 0.0
    N = len(u)
    for c in range(d, N, d):
        e = min(c + d, N)
        v[c:e] += a * v[c - d:e - d]
    return v


def render(x, rev: dict, g_reverb, predelay_s: float, crossovers, fs: float = 48000.0):
    """One source: x [N] -> q [N][K].  rev: the source's reverberator parameters
    (t_comb, g_comb [N_comb][B], comb_in [N_comb][K], J [N_comb][K][K], D [B][K][K])."""
    bands = split_bands(x, crossovers, fs)
    B = len(bands)
    N = len(x)
    K = np.asarray(rev["J"]).shape[1]
    p = delay_samples(predelay_s, fs)
    q = np.zeros((N, K))
    for b in range(B):
        xb = np.zeros(N)
        xb[p:] = bands[b][:N - p] if p < N else 0.0
        c = np.zeros((N, K))
        for i in range(len(rev["t_comb"])):
            u = xb[:, None] * np.asarray(rev["comb_in"][i])[None, :K]
            c += comb(u, float(rev["g_comb"][i][b]), rev["J"][i], max(1, delay_samples(rev["t_comb"][i], fs)))
        v = c
        for ms in AP_DELAYS_MS:
            v = allpass(v, AP_GAIN, max(1, delay_samples(ms / 1000.0, fs)))
        g = float(g_reverb[b]) if np.isfinite(g_reverb[b]) else 0.0
        q += g * (v @ np.asarray(rev["D"][b]).T)
    return q
