"""FP64 CPU oracle of the ray-parameterized reverberation hot path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product path never imports this package,
and this package never imports the product package.  Inputs come from the seeded
scene generator (a module that holds none of the method's arithmetic).

The arithmetic lives in ``oracle.c`` (plain C, double precision, built with gcc
without FMA contraction); this file only marshals arguments through ctypes.
Which paper passage each function follows is stated in ``oracle.c``.

Pins of every function against something other than itself (closed forms,
library routines, brute force, physical invariants) are in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "mlp.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

MAXB = 8
MAXK = 16
ST_COUNT = 48
EP_COUNT = 32
DIRECT_STRIDE = 21
RANGE_NAMES = {0: "none", 1: "T30", 2: "T20", 3: "T10"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, -O2, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _TraceParams(C.Structure):
    _fields_ = [
        ("num_rays", C.c_int64),
        ("max_order", C.c_int32),
        ("sh_order", C.c_int32),
        ("num_bins", C.c_int32),
        ("min_order", C.c_int32),
        ("ir_rate_hz", C.c_double),
        ("speed_of_sound", C.c_double),
        ("source_radius", C.c_double),
        ("seed", C.c_uint64),
        ("scene_id", C.c_uint32),
        ("budget_refill", C.c_int32),
        ("first_ray", C.c_int64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        P = C.POINTER
        dp, fp, ip = P(C.c_double), P(C.c_float), P(C.c_int)
        lib.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        lib.orc_sh_eval.argtypes = [C.c_int, dp, dp]
        lib.orc_intersect_tri.argtypes = [dp, dp, dp, dp, dp, dp]
        lib.orc_intersect_tri.restype = C.c_int
        lib.orc_scene_create.argtypes = [fp, C.c_int, ip, C.c_int, ip, fp, fp, C.c_int, C.c_int,
                                         C.c_double, C.c_int]
        lib.orc_scene_create.restype = C.c_void_p
        lib.orc_scene_destroy.argtypes = [C.c_void_p]
        lib.orc_scene_tmin.argtypes = [C.c_void_p]
        lib.orc_scene_tmin.restype = C.c_double
        lib.orc_scene_num_nodes.argtypes = [C.c_void_p]
        lib.orc_closest_hit.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_double, C.c_int, dp]
        lib.orc_closest_hit.restype = C.c_int
        lib.orc_any_hit.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_double, C.c_int]
        lib.orc_any_hit.restype = C.c_int
        lib.orc_trace_rays.argtypes = [C.c_void_p, P(_TraceParams), dp, dp, C.c_int, C.c_int64,
                                       C.c_int64, dp, dp, P(C.c_uint64)]
        lib.orc_trace.argtypes = [C.c_void_p, P(_TraceParams), dp, dp, C.c_int, dp, dp,
                                  P(C.c_uint64), C.c_int64]
        lib.orc_trace.restype = C.c_int
        lib.orc_direct.argtypes = [C.c_void_p, P(_TraceParams), dp, dp, C.c_int, dp]
        lib.orc_trace_ray_log.argtypes = [C.c_void_p, P(_TraceParams), dp, dp, C.c_int, C.c_uint64, dp, dp,
                                          ip, dp, dp, dp]
        lib.orc_trace_ray_log.restype = C.c_int
        lib.orc_er_rays.argtypes = [C.c_void_p, P(_TraceParams), dp, dp, C.c_int, C.c_int64, C.c_int64, dp,
                                    C.c_int64]
        lib.orc_er_rays.restype = C.c_int64
        lib.orc_next_wave.argtypes = [C.c_int64, C.c_int, C.c_double]
        lib.orc_next_wave.restype = C.c_int64
        lib.orc_estimate.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_double, dp, dp]
        lib.orc_mean_free_path.argtypes = [dp]
        lib.orc_mean_free_path.restype = C.c_double
        if hasattr(lib, "orc_mlp_forward"):
            _bind_mlp(lib)
        _lib = lib
        return lib


def _bind_mlp(lib):
    P = C.POINTER
    dp = P(C.c_double)
    lib.orc_mlp_forward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp]
    lib.orc_mlp_loss_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp,
                                      dp, dp]
    lib.orc_mlp_loss_grad.restype = C.c_double
    lib.orc_adamw_step.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_int]
    lib.orc_mlp_features.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, dp, C.c_int, dp]
    lib.orc_mlp_param_count.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    lib.orc_mlp_param_count.restype = C.c_int64


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# ----------------------------------------------------------------------------
# elementary functions
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block of counter ctr (4 x u32) under key (2 x u32)."""
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def sh_eval(order: int, direction) -> np.ndarray:
    """Real orthonormal SH (Condon-Shortley phase, ACN order) of one direction."""
    lib = _load()
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros((order + 1) ** 2, dtype=np.float64)
    lib.orc_sh_eval(order, _d(d), _d(Y))
    return Y


def intersect_tri(o, d, v0, v1, v2):
    lib = _load()
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (o, d, v0, v1, v2)]
    t = np.zeros(1)
    hit = lib.orc_intersect_tri(*[_d(a) for a in arrs], _d(t))
    return float(t[0]) if hit else None


# ----------------------------------------------------------------------------
# scene
# ----------------------------------------------------------------------------
class OracleScene:
    """The mesh and materials in double precision; use_bvh=False means brute force."""

    def __init__(self, verts, tris, tri_material, absorption, scattering, ray_eps=0.0,
                 use_bvh=None):
        lib = _load()
        self._v = np.ascontiguousarray(verts, dtype=np.float32)
        self._t = np.ascontiguousarray(tris, dtype=np.int32)
        self._m = np.ascontiguousarray(tri_material, dtype=np.int32)
        self._a = np.ascontiguousarray(absorption, dtype=np.float32)
        self._s = np.ascontiguousarray(scattering, dtype=np.float32)
        self.B = int(self._a.shape[1])
        if use_bvh is None:
            use_bvh = self._t.shape[0] > 64
        self.use_bvh = bool(use_bvh)
        self._h = lib.orc_scene_create(_f(self._v), self._v.shape[0], _i(self._t), self._t.shape[0],
                                       _i(self._m), _f(self._a), _f(self._s), self._a.shape[0],
                                       self.B, float(ray_eps), int(self.use_bvh))
        if not self._h:
            raise ValueError("oracle rejected the scene")

    @classmethod
    def from_scene(cls, sc, **kw):
        return cls(sc.verts, sc.tris, sc.tri_material, sc.absorption, sc.scattering, **kw)

    @property
    def tmin(self) -> float:
        return float(_load().orc_scene_tmin(self._h))

    def closest_hit(self, o, d, tmin=None, tmax=np.inf, exclude=-1):
        lib = _load()
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = np.zeros(1)
        tri = lib.orc_closest_hit(self._h, _d(o), _d(d), self.tmin if tmin is None else tmin,
                                  float(tmax), int(exclude), _d(t))
        return (tri, float(t[0])) if tri >= 0 else (-1, np.inf)

    def any_hit(self, o, d, tmin=None, tmax=np.inf, exclude=-1) -> bool:
        lib = _load()
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        return bool(lib.orc_any_hit(self._h, _d(o), _d(d), self.tmin if tmin is None else tmin,
                                    float(tmax), int(exclude)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_scene_destroy(self._h)
            self._h = None


# ----------------------------------------------------------------------------
# trace, direct sound, estimator
# ----------------------------------------------------------------------------
@dataclass
class TraceParams:
    num_rays: int = 10000
    max_order: int = 20
    sh_order: int = 1
    num_bins: int = 1000
    min_order: int = 1
    ir_rate_hz: float = 1000.0
    speed_of_sound: float = 343.0
    source_radius: float = 0.5
    seed: int = 0xC0FFEE
    scene_id: int = 0
    budget_refill: int = 0
    first_ray: int = 0

    def c(self) -> _TraceParams:
        return _TraceParams(int(self.num_rays), int(self.max_order), int(self.sh_order),
                            int(self.num_bins), int(self.min_order), float(self.ir_rate_hz),
                            float(self.speed_of_sound), float(self.source_radius),
                            int(self.seed) & 0xFFFFFFFFFFFFFFFF, int(self.scene_id) & 0xFFFFFFFF,
                            int(self.budget_refill), int(self.first_ray))


STAT_NAMES = {
    "escaped": (0, 8), "absorbed": (8, 16), "remaining": (16, 24), "late": (24, 32),
}
STAT_SCALARS = {
    "mfp_sum": 32, "mfp_count": 33, "mfp_sum_np": 34, "mfp_count_np": 35, "segments": 36,
    "shadow_rays": 37, "primaries": 38, "contributions": 39, "sphere_hits": 40, "waves": 41,
}


def stats_dict(st: np.ndarray, B: int) -> dict:
    out = {k: st[a:a + B].copy() for k, (a, _) in STAT_NAMES.items()}
    out.update({k: float(st[i]) for k, i in STAT_SCALARS.items()})
    out["mean_free_path"] = out["mfp_sum"] / out["mfp_count"] if out["mfp_count"] else np.nan
    out["mean_free_path_np"] = (out["mfp_sum_np"] / out["mfp_count_np"]
                                if out["mfp_count_np"] else np.nan)
    return out


def _src_arrays(listener, sources):
    lis = np.ascontiguousarray(listener, dtype=np.float64).reshape(3)
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
    return lis, src


def trace(scene: OracleScene, p: TraceParams, listener, sources, hash_cap: int = 0):
    """Single-threaded trace step.  Returns (H [S,B,K,T] float64, stats dict, hashes)."""
    lib = _load()
    lis, src = _src_arrays(listener, sources)
    S, B, K, T = src.shape[0], scene.B, (p.sh_order + 1) ** 2, p.num_bins
    H = np.zeros((S, B, K, T))
    st = np.zeros(ST_COUNT)
    hashes = np.zeros(max(hash_cap, 1), dtype=np.uint64)
    cp = p.c()
    lib.orc_trace(scene._h, C.byref(cp), _d(lis), _d(src), S, _d(H), _d(st),
                  hashes.ctypes.data_as(C.POINTER(C.c_uint64)) if hash_cap else None, int(hash_cap))
    return H, stats_dict(st, B), hashes[:hash_cap]


def trace_rays(scene: OracleScene, p: TraceParams, listener, sources, begin: int, end: int,
               want_hash: bool = False):
    """Raw (un-normalised) sums over primaries [begin, end): (H_raw, stats array, hashes)."""
    lib = _load()
    lis, src = _src_arrays(listener, sources)
    S, B, K, T = src.shape[0], scene.B, (p.sh_order + 1) ** 2, p.num_bins
    H = np.zeros((S, B, K, T))
    st = np.zeros(ST_COUNT)
    hashes = np.zeros(max(end - begin, 1), dtype=np.uint64)
    cp = p.c()
    lib.orc_trace_rays(scene._h, C.byref(cp), _d(lis), _d(src), S, int(begin), int(end), _d(H),
                       _d(st), hashes.ctypes.data_as(C.POINTER(C.c_uint64)) if want_hash else None)
    return H, st, hashes[: end - begin]


def trace_parallel(scene: OracleScene, p: TraceParams, listener, sources, threads: int = 0,
                   chunk: int = 0, hash_cap: int = 0):
    """The same step as `trace`, with each wave's primaries split into contiguous
    chunks traced by threads (ctypes releases the GIL).  Thread i traces chunks i,
    i + threads, ... of every wave into partial sums of its own, kept across the
    refill waves, and the partial sums are added in thread order at the end, so the
    result is deterministic and differs from `trace` only by FP64 rounding order."""
    threads = threads or os.cpu_count() or 1
    lis, src = _src_arrays(listener, sources)
    S, B, K, T = src.shape[0], scene.B, (p.sh_order + 1) ** 2, p.num_bins
    hashes = np.zeros(max(hash_cap, 1), dtype=np.uint64)
    begin, count, waves = int(p.first_ray), int(p.num_rays), 0
    lib = _load()
    cp = p.c()
    parts_H: list = [None] * threads
    parts_st = [np.zeros(ST_COUNT) for _ in range(threads)]
    while count > 0:
        csz = chunk or max(1, -(-count // (threads * 4)))
        ranges = [(a, min(a + csz, begin + count)) for a in range(begin, begin + count, csz)]
        used = min(threads, len(ranges))

        def worker(i):
            if parts_H[i] is None:
                parts_H[i] = np.zeros((S, B, K, T))
            for a, b in ranges[i::used]:
                a0 = a - int(p.first_ray)
                hh = None
                if hash_cap > a0 >= 0:
                    hh = np.zeros(b - a, dtype=np.uint64)
                lib.orc_trace_rays(scene._h, C.byref(cp), _d(lis), _d(src), S, int(a), int(b), _d(parts_H[i]),
                                   _d(parts_st[i]), hh.ctypes.data_as(C.POINTER(C.c_uint64)) if hh is not None
                                   else None)
                if hh is not None:
                    n = min(b - int(p.first_ray), hash_cap) - a0
                    hashes[a0:a0 + n] = hh[:n]

        ths = [threading.Thread(target=worker, args=(i,)) for i in range(used)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        begin += count
        waves += 1
        segs = sum(float(x[36]) for x in parts_st)
        count = int(lib.orc_next_wave(int(p.num_rays), int(p.max_order), segs)) if p.budget_refill else 0
    H = np.zeros((S, B, K, T))
    st = np.zeros(ST_COUNT)
    for h, x in zip(parts_H, parts_st):
        if h is not None:
            H += h
        st += x
    st[41] = waves
    kp = st[38]
    if kp > 0:
        H /= kp
        st[24:32] /= kp
    if p.min_order == 0:
        dd = direct(scene, p, lis, src)
        for s in range(S):
            if dd["visible"][s] and dd["bin"][s] < T:
                H[s, :, :, int(dd["bin"][s])] += dd["sh"][s][None, :K]
    return H, stats_dict(st, B), hashes[:hash_cap]


# ----------------------------------------------------------------------------
# Temporal coherence (Section 5): the early-reflection diffuse path cache with SH
# directivity per path, the prioritisation of early paths (the N_ER most intense are
# rendered, the rest join the late IR), and the impulse-response cache of the late IR.
# ----------------------------------------------------------------------------
ER_REC = 30
ER_NONE = -1  # triangle of reflection 2 of an order-1 path


def er_records(scene: OracleScene, p: TraceParams, listener, sources, num_primaries: int) -> np.ndarray:
    """Early-reflection contribution records [n, 30] of primaries first_ray ..
    first_ray + num_primaries - 1 (the primaries of a trace step, refill waves
    included): source, order, triangles of reflections 1 and 2, path length, ray id,
    energy per band (not divided by the primaries), SH basis of the arrival direction.
    Paths are followed with the trace step's random numbers to order min_order - 1."""
    lib = _load()
    lis, src = _src_arrays(listener, sources)
    S = src.shape[0]
    cp = p.c()
    b0, b1 = int(p.first_ray), int(p.first_ray) + int(num_primaries)
    cap = max(1, (b1 - b0) * 2 * max(S, 1))
    rec = np.zeros((cap, ER_REC))
    n = int(lib.orc_er_rays(scene._h, C.byref(cp), _d(lis), _d(src), S, b0, b1, _d(rec), cap))
    assert n <= cap
    return rec[:n]


def er_paths(scene: OracleScene, p: TraceParams, listener, sources, num_primaries: int) -> dict:
    """This update's early-reflection paths [reading of Section 5's diffuse path
    cache]: the records with the same key (source, triangle of reflection 1, triangle
    of reflection 2 or none) are one path.  Per path, over its records r, with K the
    step's primaries:
        energy[b] = sum_r e_r[b] / K
        sh[b][k]  = sum_r e_r[b] Y_k(d0_r) / K     (directivity of the path)
        delay     = sum_r E_r t_r / sum_r E_r,  E_r = sum_b e_r[b],  t_r = length_r / c
    Paths sorted by key."""
    rec = er_records(scene, p, listener, sources, num_primaries)
    B = scene.B
    K = (p.sh_order + 1) ** 2
    kp = float(num_primaries)
    out = {"source": np.zeros(0, np.int64), "tri1": np.zeros(0, np.int64), "tri2": np.zeros(0, np.int64),
           "order": np.zeros(0, np.int64), "energy": np.zeros((0, B)), "sh": np.zeros((0, B, K)),
           "delay": np.zeros(0)}
    if len(rec) == 0:
        return out
    keys = rec[:, [0, 2, 3]].astype(np.int64)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    n = len(uniq)
    e = rec[:, 6:6 + B]
    Y = rec[:, 14:14 + K]
    E = np.zeros((n, B))
    X = np.zeros((n, B, K))
    np.add.at(E, inv, e)
    np.add.at(X, inv, e[:, :, None] * Y[:, None, :])
    etot = e.sum(axis=1)
    t = rec[:, 4] / p.speed_of_sound
    num = np.zeros(n)
    den = np.zeros(n)
    np.add.at(num, inv, etot * t)
    np.add.at(den, inv, etot)
    order = np.where(uniq[:, 2] == ER_NONE, 1, 2)
    return {"source": uniq[:, 0], "tri1": uniq[:, 1], "tri2": uniq[:, 2], "order": order, "energy": E / kp,
            "sh": X / kp, "delay": np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)}


def smoothing_alpha(dt_update: float, tau: float, first: bool) -> float:
    """alpha = 1 - exp(-dt / tau) of the exponential smoothing (Section 4.2's RT60
    smoothing; Section 5 gives tau_ER = 1 s, tau_LR = 3 s); 1 on the first update or
    without smoothing (tau = 0)."""
    if first or tau <= 0.0:
        return 1.0
    return 1.0 - np.exp(-dt_update / tau)


def er_cache_update(cache: dict | None, frame: dict, alpha: float, prune: float = 0.0) -> dict:
    """The diffuse path cache [reading]: every key of the cache or of this update's
    paths is kept with
        energy = (1 - alpha) energy_cached + alpha energy_frame   (absent: zero)
        sh     = (1 - alpha) sh_cached     + alpha sh_frame
        delay  = energy-weighted mean of the two delays, weights (1 - alpha) E_cached
                 and alpha E_frame (E = sum over bands)
    and paths whose total energy falls to `prune` or below are dropped."""
    if cache is None or len(cache["source"]) == 0:
        keys = [("frame", i) for i in range(len(frame["source"]))]
        src = {"frame": frame}
        w = {"frame": alpha}
    else:
        src = {"cache": cache, "frame": frame}
        w = {"cache": 1.0 - alpha, "frame": alpha}
    table: dict = {}
    for name, d in src.items():
        for i in range(len(d["source"])):
            k = (int(d["source"][i]), int(d["tri1"][i]), int(d["tri2"][i]))
            ent = table.setdefault(k, [None, None])
            ent[0 if name == "cache" else 1] = i
    B = frame["energy"].shape[1] if len(frame["source"]) else cache["energy"].shape[1]
    K = frame["sh"].shape[2] if len(frame["source"]) else cache["sh"].shape[2]
    rows = []
    for k in sorted(table):
        ic, jf = table[k]
        E = np.zeros(B)
        X = np.zeros((B, K))
        num = den = 0.0
        for idx, name in ((ic, "cache"), (jf, "frame")):
            if idx is None or name not in src:
                continue
            d, a = src[name], w[name]
            E += a * d["energy"][idx]
            X += a * d["sh"][idx]
            et = a * d["energy"][idx].sum()
            num += et * d["delay"][idx]
            den += et
        if E.sum() <= prune:
            continue
        rows.append((k, E, X, num / den if den > 0 else 0.0))
    return {"source": np.array([r[0][0] for r in rows], np.int64), "tri1": np.array([r[0][1] for r in rows], np.int64),
            "tri2": np.array([r[0][2] for r in rows], np.int64),
            "order": np.array([1 if r[0][2] == ER_NONE else 2 for r in rows], np.int64),
            "energy": np.array([r[1] for r in rows]).reshape(-1, B), "sh": np.array([r[2] for r in rows]).reshape(-1, B, K),
            "delay": np.array([r[3] for r in rows])}


def er_prioritize(cache: dict, n_er: int = 100, hearing_threshold: float = 0.0):
    """Section 5's prioritisation: paths at or below the threshold of hearing (total
    energy over bands, per unit source power) are discarded; the rest are sorted by
    decreasing intensity (total energy; equal intensities by key) and the first
    n_er among all sources are rendered.  Returns (rendered indices in that order,
    indices of the other kept paths)."""
    n = len(cache["source"])
    if n == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    inten = cache["energy"].sum(axis=1)
    keep = np.nonzero(inten > hearing_threshold)[0]
    order = sorted(keep.tolist(), key=lambda i: (-inten[i], int(cache["source"][i]), int(cache["tri1"][i]),
                                                int(cache["tri2"][i])))
    return np.array(order[:n_er], np.int64), np.array(sorted(order[n_er:]), np.int64)


def er_spill(H, cache: dict, idx, ir_rate_hz: float) -> np.ndarray:
    """Section 5: the early paths that are not rendered are added to the late IR
    before it is analysed -- path i's SH energy sh[i] into bin floor(delay_i f_ir) of
    its source (dropped past the last bin).  Returns the new H (a copy)."""
    H = np.array(H, dtype=np.float64, copy=True)
    T = H.shape[3]
    for i in idx:
        b = int(np.floor(cache["delay"][i] * ir_rate_hz))
        if b < T:
            H[int(cache["source"][i]), :, :, b] += cache["sh"][i]
    return H


def ir_cache_update(C_prev, L, alpha: float) -> np.ndarray:
    """The impulse response cache of the late IR [reading of Section 5]: every cell of
    the SH energy histogram smoothed exponentially, C = (1 - alpha) C_prev + alpha L
    (C_prev ignored when alpha = 1)."""
    L = np.asarray(L, dtype=np.float64)
    if C_prev is None or alpha >= 1.0:
        return L.copy()
    return (1.0 - alpha) * np.asarray(C_prev, dtype=np.float64) + alpha * L


def trace_ray_log(scene: OracleScene, p: TraceParams, listener, sources, rid: int) -> dict:
    """Segments of one primary ray: triangle, t, origin and direction per segment."""
    lib = _load()
    lis, src = _src_arrays(listener, sources)
    S, B, K, T = src.shape[0], scene.B, (p.sh_order + 1) ** 2, p.num_bins
    M = max(int(p.max_order), 1)
    H = np.zeros((S, B, K, T))
    st = np.zeros(ST_COUNT)
    tri = np.zeros(M, np.int32)
    t = np.zeros(M)
    o = np.zeros((M, 3))
    d = np.zeros((M, 3))
    cp = p.c()
    n = lib.orc_trace_ray_log(scene._h, C.byref(cp), _d(lis), _d(src), S, int(rid), _d(H), _d(st), _i(tri),
                              _d(t), _d(o), _d(d))
    return {"tri": tri[:n], "t": t[:n], "o": o[:n], "d": d[:n]}


def direct(scene: OracleScene, p: TraceParams, listener, sources) -> dict:
    lib = _load()
    lis, src = _src_arrays(listener, sources)
    S = src.shape[0]
    K = (p.sh_order + 1) ** 2
    out = np.zeros((S, DIRECT_STRIDE))
    cp = p.c()
    lib.orc_direct(scene._h, C.byref(cp), _d(lis), _d(src), S, _d(out))
    return {"visible": out[:, 0] > 0, "dist": out[:, 1], "time": out[:, 2], "energy": out[:, 3],
            "bin": out[:, 4].astype(np.int64), "sh": out[:, 5:5 + K].copy()}


EP_FIELDS = ["rt60_raw", "rt60_smoothed", "fit_hi_db", "fit_lo_db", "fit_r2", "slope_db_per_s",
             "intercept_db", "i_total", "g_reverb", "e_direct", "drr_db", "predelay_s",
             "range_kind", "n_fit", "fit_j0", "fit_j1"]


def estimate(H, e_direct, ir_rate_hz: float, dt_update: float = 0.0, tau: float = 0.0,
             state=None) -> dict:
    """Reverb parameters per (source, band) from H [S,B,K,T] (float64 view taken)."""
    lib = _load()
    H = np.ascontiguousarray(H, dtype=np.float64)
    S, B, K, T = H.shape
    ed = np.ascontiguousarray(e_direct if e_direct is not None else np.zeros(S), np.float64)
    out = np.zeros((S, B, EP_COUNT))
    st = None
    if state is not None:
        st = state if (isinstance(state, np.ndarray) and state.dtype == np.float64
                       and state.flags.c_contiguous) else np.ascontiguousarray(state, np.float64)
    lib.orc_estimate(_d(H), _d(ed), S, B, K, T, float(ir_rate_hz), float(dt_update), float(tau),
                     _d(out), _d(st) if st is not None else None)
    res = {name: out[:, :, i].copy() for i, name in enumerate(EP_FIELDS)}
    res["xbar"] = out[:, :, 16:16 + K].copy()
    res["range_kind"] = res["range_kind"].astype(np.int64)
    return res


# ----------------------------------------------------------------------------
# learned estimator (oracle/mlp.c)
# ----------------------------------------------------------------------------
def mlp_param_count(din: int, dh: int, nh: int, dout: int) -> int:
    return int(_load().orc_mlp_param_count(din, dh, nh, dout))


def mlp_features(H, scene, ir_rate: float, in_dim: int = 528) -> np.ndarray:
    """Network inputs [S, in_dim] of H [S, B, K, T] and scene features [S, 10]."""
    lib = _load()
    H = np.ascontiguousarray(H, np.float64)
    S, B, K, T = H.shape
    scene = np.ascontiguousarray(scene, np.float64).reshape(S, 10)
    X = np.zeros((S, in_dim))
    lib.orc_mlp_features(S, B, K, T, float(ir_rate), _d(H), _d(scene), in_dim, _d(X))
    return X


def mlp_forward(P, X, din: int, dh: int, nh: int, dout: int) -> np.ndarray:
    lib = _load()
    P = np.ascontiguousarray(P, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, din)
    Y = np.zeros((X.shape[0], dout))
    lib.orc_mlp_forward(X.shape[0], din, dh, nh, dout, _d(P), _d(X), _d(Y))
    return Y


def mlp_loss_grad(P, X, T, mask, din: int, dh: int, nh: int, dout: int):
    """(loss, gradient in the parameter layout) of the masked mean-squared error."""
    lib = _load()
    P = np.ascontiguousarray(P, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, din)
    T = np.ascontiguousarray(T, np.float64).reshape(-1, dout)
    Mk = np.ascontiguousarray(mask, np.float64).reshape(-1, dout)
    G = np.zeros_like(P)
    loss = lib.orc_mlp_loss_grad(X.shape[0], din, dh, nh, dout, _d(P), _d(X), _d(T), _d(Mk), _d(G))
    return float(loss), G


def adamw_step(p, g, m, v, lr, beta1, beta2, eps, wd, step):
    """In-place AdamW update of float64 arrays p, m, v with gradient g."""
    lib = _load()
    g = np.ascontiguousarray(g, np.float64)
    lib.orc_adamw_step(p.size, _d(p), _d(g), _d(m), _d(v), float(lr), float(beta1), float(beta2), float(eps),
                       float(wd), int(step))


def mlp_split(P, din: int, dh: int, nh: int, dout: int):
    """List of (W [in, out], b [out]) views of a flat parameter vector."""
    out, o = [], 0
    for l in range(nh + 1):
        i = din if l == 0 else dh
        w = dout if l == nh else dh
        W = P[o:o + i * w].reshape(i, w)
        o += i * w
        b = P[o:o + w]
        o += w
        out.append((W, b))
    return out


from . import reverb  # noqa: E402,F401  (reverberator parameters, Sections 4.1-4.2)
from . import reverberator  # noqa: E402,F401  (the SH-domain Schroeder reverberator, Section 4.1)
