"""Host-side scene generators of the benchmark workloads (no GPU): the sizes they are
named for, points in free space, and determinism under their seeds."""
import numpy as np

from paper_1803_00430_gb300 import scenes


def _outside_boxes(p, boxes, margin):
    lo, hi = boxes[:, 0, :] - margin, boxes[:, 1, :] + margin
    return not np.any(np.all((p >= lo) & (p <= hi), axis=1))


def test_paper_city_has_the_papers_size():
    sc = scenes.paper_city()
    # 64 x 64 buildings x 5 faces x 5 x 5 quads x 2 triangles, plus a 64 x 64 ground grid
    assert len(sc.tris) == 64 * 64 * 5 * 5 * 5 * 2 + 64 * 64 * 2 == 1_032_192
    assert sc.num_sources == 13 and sc.num_bands == 4
    assert sc.absorption.shape == (8, 4) and np.all((sc.absorption >= 0.02) & (sc.absorption <= 0.3))


def test_city_listeners_are_distinct_free_points():
    sc = scenes.city()
    lis = scenes.city_listeners(sc, 5)
    assert lis.shape == (5, 3) and lis.dtype == np.float32
    np.testing.assert_array_equal(lis[0], sc.listener)
    pts = np.concatenate([lis, sc.sources]).astype(np.float64)
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1) + np.eye(len(pts)) * 1e9
    assert d.min() >= 1.0 - 1e-4
    for p in lis[1:].astype(np.float64):
        assert 1.0 <= p[2] <= 20.0 and 0.0 <= p[0] <= sc.room_hi[0] and 0.0 <= p[1] <= sc.room_hi[1]
        assert _outside_boxes(p, sc.boxes, 1.0 - 1e-4)
    # seeded: the same call gives the same points
    np.testing.assert_array_equal(lis, scenes.city_listeners(sc, 5))
    assert scenes.city_listeners(sc, 1).shape == (1, 3)
