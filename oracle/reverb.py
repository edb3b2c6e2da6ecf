"""FP64 oracle of the reverberator parameters (Sections 4.1 and 4.2), test
infrastructure only: the comb delays drawn from the mean free path and kept until it
moves by more than 2 sigma, the comb feedback gains, each comb's input direction
from the early IR directivity, the SH rotation matrices of the combs' feedback paths,
and the directional loudness matrices.  Plain numpy with the oracle's Philox and SH
(oracle.philox4x32_10, oracle.sh_eval); nothing here is shared with the GPU library.

Readings where the paper leaves a choice (also listed in the design doc):
  * random numbers: Philox4x32-10 with key = seed and counter (source, comb, word,
    tag); tag 2 the rotation angles (word 0), tag 3 the delays (word = draw
    generation); uniforms from the top 24 bits; normals by Box-Muller;
  * delays: mean r_free / c, sigma = mean / 3, clamped below at mean / 10;
  * rotations: R = Rz(gamma) Ry(beta) Rx(alpha), each angle uniform in [90, 270] degrees;
  * SH rotation: J(R) is the matrix with Y(R d) = J(R) Y(d) for every direction d,
    computed here by its definition J_kk' = integral of Y_k(R x) Y_k'(x) over the
    sphere (an exact product Gauss rule);
  * comb input direction: the band-summed first-order directivity of the IR at
    t_first + t_comb (t_first = the first non-zero bin over bands, bins at j / rate,
    linear interpolation, clamped to the last bin); +z when it vanishes;
  * directional loudness: the average directivity's direction density
    f(x) = sum_k xbar_k Y_k(x), amplitude gain a(x) = sqrt(max(f, 0) / f_mean) with
    f_mean = xbar_0 Y_00 (the sphere mean of f), D = sum_j w_j a(x_j) Y(x_j) Y(x_j)^T
    over a product Gauss rule (Gauss-Legendre in cos(theta) with 2n + 2 nodes times
    4n + 4 equal azimuths; the paper's spherical t-design) -- D = I when the
    reverberation is isotropic.
"""
from __future__ import annotations

import numpy as np

N_COMB = 8
TAG_ROT, TAG_DELAY = 2, 3


def _uniform(x: int) -> float:
    return (int(x) >> 8) * (1.0 / 16777216.0)


def _philox(ctr, seed: int):
    from . import philox4x32_10
    return philox4x32_10(ctr, [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])


def comb_rotation(seed: int, source: int, comb: int) -> tuple[np.ndarray, np.ndarray]:
    """The comb's random rotation: (3x3 matrix, angles (alpha, beta, gamma))."""
    r = _philox([source, comb, 0, TAG_ROT], seed)
    a = [np.pi * (0.5 + _uniform(r[i])) for i in range(3)]
    ca, sa = np.cos(a[0]), np.sin(a[0])
    cb, sb = np.cos(a[1]), np.sin(a[1])
    cg, sg = np.cos(a[2]), np.sin(a[2])
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx, np.array(a)


def sphere_rule(order: int):
    """Product Gauss rule exact for polynomials of degree <= 4 order + 3 on the sphere:
    (directions [J, 3], weights [J]) with sum of weights 4 pi."""
    nt, nphi = 2 * order + 2, 4 * order + 4
    xg, wg = np.polynomial.legendre.leggauss(nt)
    dirs, w = [], []
    for z, wz in zip(xg, wg):
        r = np.sqrt(max(0.0, 1.0 - z * z))
        for k in range(nphi):
            ph = 2.0 * np.pi * k / nphi
            dirs.append([r * np.cos(ph), r * np.sin(ph), z])
            w.append(wz * 2.0 * np.pi / nphi)
    return np.array(dirs), np.array(w)


def sh_matrix(order: int, dirs) -> np.ndarray:
    from . import sh_eval
    return np.array([sh_eval(order, d) for d in dirs])


def sh_rotation(R, order: int) -> np.ndarray:
    """J with Y(R d) = J Y(d): J = integral Y(R x) Y(x)^T dx (exact: degree 2 order)."""
    dirs, w = sphere_rule(order)
    Y = sh_matrix(order, dirs)
    YR = sh_matrix(order, dirs @ np.asarray(R).T)
    return (YR * w[:, None]).T @ Y


def directional_loudness(xbar, order: int) -> np.ndarray:
    """D for one band from its average directivity xbar [K]."""
    dirs, w = sphere_rule(order)
    Y = sh_matrix(order, dirs)
    f = Y @ np.asarray(xbar, float)
    fmean = float(xbar[0]) * 0.28209479177387814
    if not fmean > 0.0:
        return np.eye(Y.shape[1])
    a = np.sqrt(np.maximum(f, 0.0) / fmean)
    return (Y * (w * a)[:, None]).T @ Y


def draw_delays(seed: int, source: int, generation: int, mean: float) -> np.ndarray:
    sigma = mean / 3.0
    out = []
    for i in range(N_COMB):
        r = _philox([source, i, generation, TAG_DELAY], seed)
        u1 = ((int(r[0]) >> 8) + 1) * (1.0 / 16777216.0)  # (0, 1]
        u2 = _uniform(r[1])
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        out.append(max(mean + sigma * z, mean / 10.0))
    return np.array(out)


def comb_direction(H_s, t_comb: float, rate: float) -> np.ndarray:
    """Dominant direction of the early IR at t_first + t_comb (Section 4.1)."""
    I = H_s[:, 0, :].sum(axis=0)
    nz = np.nonzero(I > 0)[0]
    T = H_s.shape[2]
    if len(nz) == 0 or H_s.shape[1] < 4:
        return np.array([0.0, 0.0, 1.0])
    x = min((nz[0] / rate + t_comb) * rate, T - 1.0)
    j0 = int(np.floor(x))
    j1 = min(j0 + 1, T - 1)
    f = x - j0
    X = H_s[:, 1:4, :].sum(axis=0)  # band-summed first-order coefficients [3][T]
    v = (1.0 - f) * X[:, j0] + f * X[:, j1]  # (X_1-1, X_10, X_11)
    d = np.array([-v[2], -v[0], v[1]])
    n = np.linalg.norm(d)
    return d / n if n > 0 else np.array([0.0, 0.0, 1.0])


def configure(H, rt60, xbar, mean_free_path: float, speed_of_sound: float, rate: float, seed: int, state=None):
    """Reverberator parameters of every source.

    H [S][B][K][T] the IR, rt60 [S][B] (the smoothed decay times), xbar [S][B][K];
    state: list of per-source dicts {mean, generation} or None (first update).
    Returns (list of per-source parameter dicts, new state)."""
    H = np.asarray(H, float)
    S, B, K, T = H.shape
    order = int(round(np.sqrt(K))) - 1
    mean = mean_free_path / speed_of_sound
    out, new_state = [], []
    for s in range(S):
        st = None if state is None else state[s]
        if st is None or st["generation"] == 0 or abs(mean - st["mean"]) > 2.0 * st["mean"] / 3.0:
            gen = 1 if st is None else st["generation"] + 1
            mu = mean
            resampled = True
        else:
            gen, mu, resampled = st["generation"], st["mean"], False
        t = draw_delays(seed, s, gen, mu)
        g = np.array([[10.0 ** (-3.0 * t[i] / rt60[s][b]) if rt60[s][b] > 0 else 0.0 for b in range(B)]
                      for i in range(N_COMB)])
        dirs = np.array([comb_direction(H[s], t[i], rate) for i in range(N_COMB)])
        from . import sh_eval
        comb_in = np.array([sh_eval(order, d) / N_COMB for d in dirs])
        rots = [comb_rotation(seed, s, i) for i in range(N_COMB)]
        J = np.array([sh_rotation(R, order) for R, _ in rots])
        D = np.array([directional_loudness(xbar[s][b], order) for b in range(B)])
        out.append({"mean_delay": mu, "generation": gen, "resampled": resampled, "t_comb": t, "g_comb": g,
                    "dir": dirs, "comb_in": comb_in, "rot": np.array([R for R, _ in rots]),
                    "angles": np.array([a for _, a in rots]), "J": J, "D": D})
        new_state.append({"mean": mu, "generation": gen})
    return out, new_state
