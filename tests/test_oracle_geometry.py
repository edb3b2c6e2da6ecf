"""Pins of the oracle's ray/triangle test, BVH and visibility.

* Moller-Trumbore against numpy's linear solve of o + t d = v0 + u e1 + v e2
  (a library routine), including edge and parallel cases.
* BVH closest-hit and any-hit against the brute-force loop on random tiny meshes
  (identical results: same double arithmetic, the BVH must only prune safely).
* Closest hit in a shoebox against the closed-form slab distance.
"""
import numpy as np

from paper_1803_00430_gb300 import scenes


def _solve_ref(o, d, v0, v1, v2):
    A = np.column_stack([-d, v1 - v0, v2 - v0])
    if abs(np.linalg.det(A)) < 1e-14:
        return None
    t, u, v = np.linalg.solve(A, o - v0)
    if u < -1e-12 or v < -1e-12 or u + v > 1 + 1e-12:
        return None
    return t


def test_moller_trumbore_matches_linear_solve(oracle_lib):
    rng = np.random.default_rng(3)
    n_hit = 0
    for _ in range(3000):
        v0, v1, v2 = rng.normal(size=(3, 3))
        o = rng.normal(size=3) * 3
        target = v0 + rng.uniform(-0.2, 1.2) * (v1 - v0) + rng.uniform(-0.2, 1.2) * (v2 - v0)
        d = target - o
        d /= np.linalg.norm(d)
        got = oracle_lib.intersect_tri(o, d, v0, v1, v2)
        ref = _solve_ref(o, d, v0, v1, v2)
        if ref is None or got is None:
            # only disagreement allowed: a hit within rounding of an edge
            if (ref is None) != (got is None):
                A = np.column_stack([-d, v1 - v0, v2 - v0])
                _, u, v = np.linalg.solve(A, o - v0)
                assert min(u, v, 1 - u - v) > -1e-9 and min(abs(u), abs(v), abs(1 - u - v)) < 1e-9
            continue
        n_hit += 1
        assert got == __import__("pytest").approx(ref, rel=1e-10, abs=1e-12)
    assert n_hit > 500


def test_parallel_ray_misses(oracle_lib):
    v0, v1, v2 = np.array([0., 0, 0]), np.array([1., 0, 0]), np.array([0., 1, 0])
    assert oracle_lib.intersect_tri([0.2, 0.2, 1], [1, 0, 0], v0, v1, v2) is None
    assert oracle_lib.intersect_tri([0.2, 0.2, 1], [0, 0, -1], v0, v1, v2) == 1.0
    # two-sided: from below
    assert oracle_lib.intersect_tri([0.2, 0.2, -2], [0, 0, 1], v0, v1, v2) == 2.0


def _random_mesh(rng, n):
    c = rng.uniform(-5, 5, size=(n, 1, 3))
    v = (c + rng.normal(scale=1.0, size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    t = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return v, t


def test_bvh_matches_brute_force(oracle_lib):
    rng = np.random.default_rng(11)
    for trial in range(4):
        n = [16, 37, 64, 64][trial]
        v, t = _random_mesh(rng, n)
        m = np.zeros(n, np.int32)
        a = np.full((1, 1), 0.1, np.float32)
        brute = oracle_lib.OracleScene(v, t, m, a, a, use_bvh=False)
        bvh = oracle_lib.OracleScene(v, t, m, a, a, use_bvh=True)
        for _ in range(2500):
            o = rng.uniform(-8, 8, size=3)
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            ex = int(rng.integers(-1, n))
            tmax = float(rng.choice([np.inf, rng.uniform(0.5, 10)]))
            r1 = brute.closest_hit(o, d, tmax=tmax, exclude=ex)
            r2 = bvh.closest_hit(o, d, tmax=tmax, exclude=ex)
            assert r1 == r2
            assert brute.any_hit(o, d, tmax=tmax, exclude=ex) == bvh.any_hit(o, d, tmax=tmax,
                                                                               exclude=ex)


def test_shoebox_closest_hit_is_slab_distance(oracle_lib):
    sc = scenes.shoebox()
    osc = oracle_lib.OracleScene.from_scene(sc)
    size = np.array([10.0, 8.0, 4.0])
    rng = np.random.default_rng(5)
    for _ in range(500):
        o = rng.uniform(0.1, size - 0.1)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tri, t = osc.closest_hit(o, d)
        ts = np.where(d > 0, (size - o) / d, -o / d)
        assert tri >= 0
        assert t == __import__("pytest").approx(ts.min(), rel=1e-12)
        # the face hit is the one of the nearest slab: faces are ordered x-lo, x-hi, ...
        ax = int(np.argmin(ts))
        face = 2 * ax + (1 if d[ax] > 0 else 0)
        assert tri // 2 == face


def test_any_hit_occlusion(oracle_lib):
    # a box between two points blocks; moving one point aside unblocks
    v, t = scenes.box_mesh([4, 4, 0], [6, 6, 3])
    m = np.zeros(12, np.int32)
    a = np.full((1, 2), 0.1, np.float32)
    osc = oracle_lib.OracleScene(v.astype(np.float32), t.astype(np.int32), m, a, a)
    p, q = np.array([1.0, 5.0, 1.0]), np.array([9.0, 5.0, 1.0])
    d = (q - p) / np.linalg.norm(q - p)
    assert osc.any_hit(p, d, tmax=np.linalg.norm(q - p))
    q2 = np.array([9.0, 9.0, 1.0])
    d2 = (q2 - p) / np.linalg.norm(q2 - p)
    assert not osc.any_hit(p, d2, tmax=np.linalg.norm(q2 - p))
    # tmax before the box: not blocked
    assert not osc.any_hit(p, d, tmax=2.0)


def test_coplanar_overlapping_triangles_tie_to_the_smaller_index(oracle_lib):
    """Two triangles with different vertices in one plane, overlapping: a ray meets both
    at one mathematical distance, so the smaller triangle index must win whatever the
    FP64 rounding of the two computed distances and whatever order the triangles are
    visited in (BVH and brute force, and both index assignments).  Lifted by 1e-5 m
    towards the rays, the second one is simply nearer."""
    rng = np.random.default_rng(12)
    a = np.array([[0.3, 0.1, 0.2], [7.9, 0.7, 0.2], [1.1, 6.3, 0.2]])
    b = np.array([[0.05, 0.4, 0.2], [6.7, -0.3, 0.2], [2.2, 7.1, 0.2]])
    for first, second, lift, want in ((a, b, 0.0, 0), (b, a, 0.0, 0), (a, b, 1e-5, 1), (b, a, 1e-5, 1)):
        s = second.copy()
        s[:, 2] += lift  # the second triangle above the first: nearer for rays from above
        verts = np.concatenate([first, s]).astype(np.float32)
        tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
        mats = np.zeros(2, np.int32)
        al = np.full((1, 1), 0.1, np.float32)
        for use_bvh in (True, False):
            osc = oracle_lib.OracleScene(verts, tris, mats, al, al, use_bvh=use_bvh)
            hits = 0
            for _ in range(400):
                p = np.array([rng.uniform(1.5, 3.5), rng.uniform(1.0, 3.0), 0.2])  # inside both
                o = p + rng.uniform(0.5, 3.0) * np.array([rng.normal(0.3, 0.2), rng.normal(0.3, 0.2), 1.0])
                d = (p - o) / np.linalg.norm(p - o)
                tri, t = osc.closest_hit(o, d)
                assert tri == want, (tri, want, lift, use_bvh)
                hits += 1
            assert hits == 400
