"""Seeded synthetic workloads: triangle meshes, materials, sources and listeners.

This module only builds inputs.  It holds none of the method's arithmetic (no
ray tracing, no energy, no spherical harmonics), so both the CUDA path and the
CPU oracle can be fed from it without sharing any computation.

The paper's own scenes (City, Hospital, Space Station, Sub Bay, Tuscany; Table 1)
are not available, so procedural stand-ins with comparable triangle and source
counts are generated here:

* ``shoebox``         -- 10 x 8 x 4 m room, 12 triangles, 4 bands, 1 source.
* ``furnished_hall``  -- 40 x 30 x 12 m hall plus 2000 seeded boxes
                         (24,012 triangles), 8 bands, 16 sources.
* ``room_or_corridor``-- a room (box + interior boxes) or a corridor (long box +
                         side rooms) of a requested triangle count (batched and
                         learned workloads).
* ``city``            -- grid of extruded tessellated buildings plus a
                         tessellated ground plane (~2M triangles).

Materials carry one absorption and one scattering coefficient per frequency band
(Section 5 uses 4 log-spaced bands).  Every generator is deterministic in its seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x5EED0000

# Seeds of the named workloads: SEED_BASE + index.
SEED_TINY = SEED_BASE + 0
SEED_MEDIUM = SEED_BASE + 1
SEED_BATCHED = SEED_BASE + 2
SEED_LEARNED = SEED_BASE + 3
SEED_LARGE = SEED_BASE + 4

# Philox key of update u is PHILOX_KEY_BASE + u.
PHILOX_KEY_BASE = 0xC0FFEE


@dataclass
class Scene:
    """A triangle mesh with per-band materials, one listener and S sources.

    verts        float32 [V, 3]   metres
    tris         int32   [T, 3]   vertex indices (two-sided surfaces; winding unused)
    tri_material int32   [T]      material index of each triangle
    absorption   float32 [Mat, B] per-band absorption coefficient alpha in [0, 1]
    scattering   float32 [Mat, B] per-band scattering coefficient s in [0, 1]
    listener     float32 [3]
    sources      float32 [S, 3]
    boxes        float64 [nb, 2, 3] axis-aligned solid boxes (lo, hi) used to place
                 points in free space; metadata only.
    """

    name: str
    verts: np.ndarray
    tris: np.ndarray
    tri_material: np.ndarray
    absorption: np.ndarray
    scattering: np.ndarray
    listener: np.ndarray
    sources: np.ndarray
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 2, 3)))
    room_lo: np.ndarray = field(default_factory=lambda: np.zeros(3))
    room_hi: np.ndarray = field(default_factory=lambda: np.zeros(3))

    @property
    def num_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def num_bands(self) -> int:
        return int(self.absorption.shape[1])

    @property
    def num_sources(self) -> int:
        return int(self.sources.shape[0])


class _MeshBuilder:
    def __init__(self):
        self.verts: list[np.ndarray] = []
        self.tris: list[np.ndarray] = []
        self.mats: list[np.ndarray] = []
        self.nv = 0

    def add(self, verts: np.ndarray, tris: np.ndarray, material: int) -> None:
        self.verts.append(np.asarray(verts, dtype=np.float64))
        self.tris.append(np.asarray(tris, dtype=np.int64) + self.nv)
        self.mats.append(np.full(len(tris), material, dtype=np.int32))
        self.nv += len(verts)

    def add_box(self, lo, hi, material: int) -> None:
        v, t = box_mesh(lo, hi)
        self.add(v, t, material)

    def finish(self):
        verts = np.concatenate(self.verts).astype(np.float32)
        tris = np.concatenate(self.tris).astype(np.int32)
        mats = np.concatenate(self.mats).astype(np.int32)
        return verts, tris, mats


def box_mesh(lo, hi):
    """8 corners and 12 triangles (2 per face) of the axis-aligned box [lo, hi]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = np.array([[lo[0] if i & 1 == 0 else hi[0],
                   lo[1] if i & 2 == 0 else hi[1],
                   lo[2] if i & 4 == 0 else hi[2]] for i in range(8)])
    faces = [  # quads as corner indices
        (0, 2, 6, 4), (1, 5, 7, 3),   # x = lo, x = hi
        (0, 4, 5, 1), (2, 3, 7, 6),   # y = lo, y = hi
        (0, 1, 3, 2), (4, 6, 7, 5),   # z = lo, z = hi
    ]
    tris = []
    for a, b, cc, d in faces:
        tris.append((a, b, cc))
        tris.append((a, cc, d))
    return c, np.array(tris, dtype=np.int64)


def grid_quad_mesh(origin, du, dv, nu: int, nv: int):
    """A planar parallelogram origin + [0,1]du + [0,1]dv tessellated into nu x nv quads."""
    origin = np.asarray(origin, dtype=np.float64)
    du = np.asarray(du, dtype=np.float64)
    dv = np.asarray(dv, dtype=np.float64)
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
    verts = origin + (ii[..., None] / nu) * du + (jj[..., None] / nv) * dv
    verts = verts.reshape(-1, 3)
    idx = lambda i, j: i * (nv + 1) + j  # noqa: E731
    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    return verts, np.array(tris, dtype=np.int64)


def _materials(rng, n_mat: int, bands: int, a_lo=0.05, a_hi=0.4, s_lo=0.1, s_hi=0.9, s_spread=None):
    """Per-band absorption U[a_lo, a_hi].  Scattering U[s_lo, s_hi] drawn per band, or,
    with s_spread set, a base value plus a rise of at most s_spread linear over the
    bands (scattering of real surfaces grows smoothly with frequency)."""
    absorption = rng.uniform(a_lo, a_hi, size=(n_mat, bands)).astype(np.float32)
    if s_spread is None:
        scattering = rng.uniform(s_lo, s_hi, size=(n_mat, bands)).astype(np.float32)
    else:
        base = rng.uniform(s_lo, s_hi - s_spread, size=(n_mat, 1))
        rise = rng.uniform(0.0, s_spread, size=(n_mat, 1))
        ramp = np.linspace(0.0, 1.0, bands)[None, :] if bands > 1 else np.zeros((1, 1))
        scattering = (base + rise * ramp).astype(np.float32)
    return absorption, scattering


def _inside_any(p, boxes, margin):
    if len(boxes) == 0:
        return False
    lo = boxes[:, 0, :] - margin
    hi = boxes[:, 1, :] + margin
    return bool(np.any(np.all((p >= lo) & (p <= hi), axis=1)))


def _free_points(rng, n, lo, hi, boxes, margin_wall, margin_box, min_sep=1.0,
                 avoid=(), max_tries=200000):
    """n points uniform in [lo+margin_wall, hi-margin_wall], outside every box grown by
    margin_box and at least min_sep from each other and from the points in `avoid`."""
    lo = np.asarray(lo, dtype=np.float64) + margin_wall
    hi = np.asarray(hi, dtype=np.float64) - margin_wall
    pts: list[np.ndarray] = []
    others = [np.asarray(a, dtype=np.float64) for a in avoid]
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place points in free space")
        p = rng.uniform(lo, hi)
        if _inside_any(p, boxes, margin_box):
            continue
        if any(np.linalg.norm(p - q) < min_sep for q in pts + others):
            continue
        pts.append(p)
    return np.array(pts)


def shoebox(seed: int = SEED_TINY, bands: int = 4, num_sources: int = 1,
            size=(10.0, 8.0, 4.0), absorption=None, scattering=None) -> Scene:
    """Tiny workload: shoebox room, 12 triangles; each pair of opposite walls shares
    one material (alpha_b ~ U[0.05,0.4], s_b ~ U[0.1,0.9]).  Source and listener are
    uniform in the room at least 0.5 m from every wall and 1 m apart."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.asarray(size, dtype=np.float64)
    v, t = box_mesh(lo, hi)
    # faces come in the order x-lo, x-hi, y-lo, y-hi, z-lo, z-hi (2 triangles each)
    mats = np.repeat(np.array([0, 0, 1, 1, 2, 2], dtype=np.int32), 2)
    a, s = _materials(rng, 3, bands)
    if absorption is not None:
        a = np.broadcast_to(np.asarray(absorption, np.float32), (3, bands)).copy()
    if scattering is not None:
        s = np.broadcast_to(np.asarray(scattering, np.float32), (3, bands)).copy()
    pts = _free_points(rng, 1 + num_sources, lo, hi, np.zeros((0, 2, 3)), 0.5, 0.0)
    return Scene("shoebox", v.astype(np.float32), t.astype(np.int32), mats, a, s,
                 pts[0].astype(np.float32), pts[1:].astype(np.float32),
                 room_lo=lo, room_hi=hi)


def furnished_hall(seed: int = SEED_MEDIUM, n_boxes: int = 2000, bands: int = 8,
                   num_sources: int = 16, size=(40.0, 30.0, 12.0)) -> Scene:
    """Medium workload: 40 x 30 x 12 m hall plus n_boxes seeded axis-aligned boxes
    (sizes U[0.3,3] m per axis, centres uniform in the hall, clipped to it; a box rests
    on the floor with probability 0.6, otherwise floats).  8 materials; box i uses
    material i mod 8, the hall uses material 0.  Sources and listener sit in free
    space (0.6 m clear of every box, 0.5 m from the walls)."""
    rng = np.random.default_rng(seed)
    size = np.asarray(size, dtype=np.float64)
    mb = _MeshBuilder()
    mb.add_box(np.zeros(3), size, 0)
    boxes = np.zeros((n_boxes, 2, 3))
    for i in range(n_boxes):
        ext = rng.uniform(0.3, 3.0, size=3)
        c = rng.uniform(np.zeros(3), size)
        lo = c - ext / 2
        hi = c + ext / 2
        if rng.uniform() < 0.6:
            lo[2] = 0.0
            hi[2] = ext[2]
        else:
            z0 = rng.uniform(0.0, size[2] - ext[2])
            lo[2], hi[2] = z0, z0 + ext[2]
        lo = np.clip(lo, 0.0, size)
        hi = np.clip(hi, 0.0, size)
        boxes[i, 0], boxes[i, 1] = lo, hi
        mb.add_box(lo, hi, i % 8)
    verts, tris, mats = mb.finish()
    a, s = _materials(rng, 8, bands)
    pts = _free_points(rng, 1 + num_sources, np.zeros(3), size, boxes, 0.5, 0.6)
    return Scene("furnished_hall", verts, tris, mats, a, s,
                 pts[0].astype(np.float32), pts[1:].astype(np.float32), boxes=boxes,
                 room_lo=np.zeros(3), room_hi=size)


def room_or_corridor(seed: int, target_tris: int, bands: int = 8, num_sources: int = 1,
                     kind: str | None = None, n_mat: int = 8, s_spread: float | None = None) -> Scene:
    """Batched / learned workload: either a room (outer box plus interior boxes) or a
    corridor (a long box with side rooms opened into it by box 'walls'), with about
    target_tris triangles (at least 12).  s_spread: see _materials."""
    rng = np.random.default_rng(seed)
    if kind is None:
        kind = "room" if rng.uniform() < 0.5 else "corridor"
    n_inner = max(0, (int(target_tris) - 12) // 12)
    boxes = []  # interior boxes (lo, hi, material)
    if kind == "room":
        size = rng.uniform([4.0, 4.0, 2.5], [30.0, 25.0, 10.0])
        for i in range(n_inner):
            ext = rng.uniform(0.2, 0.25 * size.min() + 0.3, size=3)
            c = rng.uniform(np.zeros(3), size)
            lo, hi = np.clip(c - ext / 2, 0, size), np.clip(c + ext / 2, 0, size)
            if rng.uniform() < 0.6:
                lo[2], hi[2] = 0.0, min(ext[2], size[2])
            boxes.append((lo, hi, 1 + i % (n_mat - 1)))
    else:
        length = rng.uniform(20.0, 80.0)
        width = rng.uniform(2.0, 5.0)
        height = rng.uniform(2.5, 5.0)
        size = np.array([length, width, height])
        # interior "side rooms": thin partition boxes that split the corridor into
        # alcoves along one side, plus clutter for the rest of the triangle budget
        for i in range(n_inner):
            if i % 2 == 0:
                x = rng.uniform(0.0, length)
                t = rng.uniform(0.1, 0.3)
                depth = rng.uniform(0.3, 0.5) * width
                side = rng.integers(0, 2)
                y0 = 0.0 if side == 0 else width - depth
                lo = np.array([max(0.0, x - t / 2), y0, 0.0])
                hi = np.array([min(length, x + t / 2), y0 + depth, height])
            else:
                ext = rng.uniform(0.2, min(1.5, 0.45 * width), size=3)
                c = rng.uniform(np.zeros(3), size)
                lo, hi = np.clip(c - ext / 2, 0, size), np.clip(c + ext / 2, 0, size)
            boxes.append((lo, hi, 1 + i % (n_mat - 1)))
    a, s = _materials(rng, n_mat, bands, s_spread=s_spread)
    margin = min(0.5, 0.2 * float(size.min()))
    min_sep = min(1.0, 0.3 * float(size.min()))
    bx = np.array([(lo, hi) for lo, hi, _ in boxes]).reshape(-1, 2, 3)
    try:
        pts = _free_points(rng, 1 + num_sources, np.zeros(3), size, bx, margin, 0.3, min_sep=min_sep,
                           max_tries=20000)
    except RuntimeError:
        # the clutter fills the room: place the points first (apart from each other) and
        # drop the boxes that would enclose one of them
        frng = np.random.default_rng([seed, 1])
        pts = _free_points(frng, 1 + num_sources, np.zeros(3), size, np.zeros((0, 2, 3)), margin, 0.3,
                           min_sep=min_sep)
        boxes = [b for b in boxes if not any(_inside_any(p, np.array([b[:2]]), 0.3) for p in pts)]
        bx = np.array([(lo, hi) for lo, hi, _ in boxes]).reshape(-1, 2, 3)
    mb = _MeshBuilder()
    mb.add_box(np.zeros(3), size, 0)
    for lo, hi, m in boxes:
        mb.add_box(lo, hi, m)
    verts, tris, mats = mb.finish()
    return Scene(f"{kind}", verts, tris, mats, a, s, pts[0].astype(np.float32),
                 pts[1:].astype(np.float32), boxes=bx, room_lo=np.zeros(3),
                 room_hi=size)


def city(seed: int = SEED_LARGE, grid: int = 64, tess: int = 7, ground_tess: int = 64,
         bands: int = 8, num_sources: int = 256, block: float = 50.0) -> Scene:
    """Large workload: grid x grid buildings (footprints U[10,40] m, heights U[5,60] m)
    on a block-spaced grid; each wall and roof is a tess x tess quad grid, and the
    ground plane a ground_tess x ground_tess grid.  Absorption U[0.02,0.3]."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    extent = grid * block
    v, t = grid_quad_mesh([0, 0, 0], [extent, 0, 0], [0, extent, 0], ground_tess,
                          ground_tess)
    mb.add(v, t, 0)
    boxes = []
    for gx in range(grid):
        for gy in range(grid):
            fx, fy = rng.uniform(10.0, 40.0, size=2)
            h = rng.uniform(5.0, 60.0)
            cx, cy = (gx + 0.5) * block, (gy + 0.5) * block
            lo = np.array([cx - fx / 2, cy - fy / 2, 0.0])
            hi = np.array([cx + fx / 2, cy + fy / 2, h])
            boxes.append((lo, hi))
            m = 1 + (gx * grid + gy) % 7
            x0, y0, _ = lo
            x1, y1, z1 = hi
            faces = [
                ([x0, y0, 0], [x1 - x0, 0, 0], [0, 0, z1]),
                ([x1, y0, 0], [0, y1 - y0, 0], [0, 0, z1]),
                ([x1, y1, 0], [x0 - x1, 0, 0], [0, 0, z1]),
                ([x0, y1, 0], [0, y0 - y1, 0], [0, 0, z1]),
                ([x0, y0, z1], [x1 - x0, 0, 0], [0, y1 - y0, 0]),
            ]
            for o, du, dv in faces:
                fv, ft = grid_quad_mesh(o, du, dv, tess, tess)
                mb.add(fv, ft, m)
    verts, tris, mats = mb.finish()
    boxes = np.array(boxes)
    a, s = _materials(rng, 8, bands, a_lo=0.02, a_hi=0.3)
    lo = np.array([0.0, 0.0, 1.0])
    hi = np.array([extent, extent, 20.0])
    pts = _free_points(rng, 1 + num_sources, lo, hi, boxes, 0.0, 1.0, min_sep=1.0)
    return Scene("city", verts, tris, mats, a, s, pts[0].astype(np.float32),
                 pts[1:].astype(np.float32), boxes=boxes, room_lo=np.zeros(3),
                 room_hi=np.array([extent, extent, 60.0]))


def paper_city(seed: int = SEED_LARGE + 2) -> Scene:
    """The paper's operating point on a city-like scene: the procedural city with 5 x 5
    quads per face (1,032,192 triangles, against the paper's City of 1,001,860), 4 bands
    and 13 sources."""
    return city(seed=seed, tess=5, bands=4, num_sources=13)


def city_listeners(sc: Scene, n: int, seed: int = SEED_LARGE + 1) -> np.ndarray:
    """n listener positions for the city: its own listener, then seeded free points
    (1-20 m above the ground, at least 1 m from buildings, sources and each other)."""
    if n <= 1:
        return sc.listener[None, :].astype(np.float32)
    rng = np.random.default_rng(seed)
    lo = np.array([0.0, 0.0, 1.0])
    hi = np.array([sc.room_hi[0], sc.room_hi[1], 20.0])
    extra = _free_points(rng, n - 1, lo, hi, sc.boxes, 0.0, 1.0, min_sep=1.0,
                         avoid=[sc.listener, *sc.sources])
    return np.concatenate([sc.listener[None, :], extra]).astype(np.float32)


def batched_specs(seed: int = SEED_BATCHED, n_scenes: int = 512, bands: int = 8):
    """Per-scene sizes of the batched workload: triangle count log-uniform in
    [12, 40k], source count log-uniform over 1..64, ray count log-uniform in
    [1e4, 3e5].  Returns a list of (scene_seed, tris, sources, rays)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        tris = int(np.exp(rng.uniform(np.log(12), np.log(40000))))
        srcs = int(np.clip(np.floor(np.exp(rng.uniform(0, np.log(65)))), 1, 64))
        rays = int(np.exp(rng.uniform(np.log(1e4), np.log(3e5))))
        out.append((seed * 1000 + i, tris, srcs, rays))
    return out
