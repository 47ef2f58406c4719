"""Seeded synthetic scenes: boxes, walls and a ground plane inside the unit cube.

The participating medium fills the unit cube [0,1]^3; all geometry lies inside
or on it (boxes are clipped to the cube).  Triangles are stored as a soup,
float32 array of shape [n_tris, 3, 3] (triangle, corner, xyz), with a
per-triangle RGB albedo and an optional per-triangle RGB emission.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Medium:
    """Homogeneous medium: scattering and absorption coefficients, HG asymmetry g."""
    sigma_s: float
    sigma_a: float
    g: float

    @property
    def sigma_t(self) -> float:
        return float(np.float32(self.sigma_s) + np.float32(self.sigma_a))


@dataclass
class PointLight:
    pos: tuple
    intensity: tuple


@dataclass
class Scene:
    tris: np.ndarray                 # float32 [n, 3, 3]
    albedo: np.ndarray               # float32 [n, 3]
    medium: Medium
    lights: List[PointLight]
    emission: Optional[np.ndarray] = None   # float32 [n, 3] or None
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 2, 3), np.float32))
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def light_arrays(self):
        pos = np.array([l.pos for l in self.lights], np.float32).reshape(-1, 3)
        inten = np.array([l.intensity for l in self.lights], np.float32).reshape(-1, 3)
        return pos, inten

    def vertex_index_form(self):
        """Return (verts [3n,3] float32, idx [n,3] int32): the soup as indexed triangles."""
        n = self.n_tris
        verts = np.ascontiguousarray(self.tris.reshape(n * 3, 3), dtype=np.float32)
        idx = np.arange(n * 3, dtype=np.int32).reshape(n, 3)
        return verts, idx


def box_triangles(lo, hi) -> np.ndarray:
    """12 triangles of an axis-aligned box, wound so normals point outward."""
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    c = np.array([[lo[0], lo[1], lo[2]], [hi[0], lo[1], lo[2]], [hi[0], hi[1], lo[2]],
                  [lo[0], hi[1], lo[2]], [lo[0], lo[1], hi[2]], [hi[0], lo[1], hi[2]],
                  [hi[0], hi[1], hi[2]], [lo[0], hi[1], hi[2]]], np.float32)
    faces = [(0, 3, 2), (0, 2, 1),      # z = lo
             (4, 5, 6), (4, 6, 7),      # z = hi
             (0, 1, 5), (0, 5, 4),      # y = lo
             (3, 7, 6), (3, 6, 2),      # y = hi
             (0, 4, 7), (0, 7, 3),      # x = lo
             (1, 2, 6), (1, 6, 5)]      # x = hi
    return np.stack([c[list(f)] for f in faces]).astype(np.float32)


def box_triangles_tessellated(lo, hi, n: int) -> np.ndarray:
    """An axis-aligned box with every face split into an n x n grid of quads (2 triangles
    each): 12 n^2 triangles, normals outward."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    out = []
    for ax in range(3):
        u, v = [a for a in range(3) if a != ax]
        for side in (0, 1):
            g = np.linspace(0.0, 1.0, n + 1)
            P = np.zeros((n + 1, n + 1, 3))
            P[..., ax] = hi[ax] if side else lo[ax]
            P[..., u] = lo[u] + (hi[u] - lo[u]) * g[:, None]
            P[..., v] = lo[v] + (hi[v] - lo[v]) * g[None, :]
            a, b, c, d = P[:-1, :-1], P[1:, :-1], P[1:, 1:], P[:-1, 1:]
            t1 = np.stack([a, b, c], axis=2).reshape(-1, 3, 3)
            t2 = np.stack([a, c, d], axis=2).reshape(-1, 3, 3)
            tri = np.concatenate([t1, t2])
            # wind outward: the normal must point along +ax on the hi side, -ax on the lo side
            nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])[:, ax]
            flip = (nrm < 0) if side else (nrm > 0)
            tri[flip] = tri[flip][:, [0, 2, 1]]
            out.append(tri)
    return np.concatenate(out).astype(np.float32)


def ground_grid(m: int) -> np.ndarray:
    """Ground plane z = 0 over [0,1]^2 as an m x m grid of quads (2 m^2 triangles)."""
    g = np.linspace(0.0, 1.0, m + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X, Y, np.zeros_like(X)], axis=-1)
    a, b, c, d = P[:-1, :-1], P[1:, :-1], P[1:, 1:], P[:-1, 1:]
    return np.concatenate([np.stack([a, b, c], 2).reshape(-1, 3, 3),
                           np.stack([a, c, d], 2).reshape(-1, 3, 3)]).astype(np.float32)


def cube_walls() -> np.ndarray:
    """The six faces of the unit cube as 12 triangles (the room of the small workload)."""
    return box_triangles((0, 0, 0), (1, 1, 1))


def ground_quads(n_tris: int) -> np.ndarray:
    """Ground plane z=0 over [0,1]^2 split into n_tris triangles (4 or 8)."""
    if n_tris == 8:
        tris = []
        for ix in range(2):
            for iy in range(2):
                x0, x1, y0, y1 = ix * 0.5, ix * 0.5 + 0.5, iy * 0.5, iy * 0.5 + 0.5
                tris.append([[x0, y0, 0], [x1, y0, 0], [x1, y1, 0]])
                tris.append([[x0, y0, 0], [x1, y1, 0], [x0, y1, 0]])
        return np.array(tris, np.float32)
    if n_tris == 4:
        c = [0.5, 0.5, 0.0]
        corners = [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]]
        return np.array([[c, corners[i], corners[(i + 1) % 4]] for i in range(4)], np.float32)
    raise ValueError("ground_quads supports 4 or 8 triangles")


def random_boxes(rng: np.random.Generator, n_boxes: int, side_lo: float, side_hi: float,
                 log_uniform: bool, keep_clear: List[np.ndarray], clear_radius: float) -> np.ndarray:
    """Axis-aligned boxes with centres U[0,1]^3, clipped to the unit cube.

    Boxes whose (clipped) extent comes within `clear_radius` of any point in
    `keep_clear` (the light position) are redrawn, so no light sits inside geometry.
    Returns float32 [n_boxes, 2, 3] (lo, hi).
    """
    out = np.zeros((n_boxes, 2, 3), np.float32)
    k = 0
    while k < n_boxes:
        if log_uniform:
            side = np.exp(rng.uniform(np.log(side_lo), np.log(side_hi), size=3))
        else:
            side = rng.uniform(side_lo, side_hi, size=3)
        ctr = rng.uniform(0.0, 1.0, size=3)
        lo = np.clip(ctr - side / 2, 0.0, 1.0).astype(np.float32)
        hi = np.clip(ctr + side / 2, 0.0, 1.0).astype(np.float32)
        if np.any(hi - lo < 1e-4):
            continue
        bad = False
        for p in keep_clear:
            d = np.maximum(np.maximum(lo - p, p - hi), 0.0)
            if float(np.sqrt((d * d).sum())) < clear_radius:
                bad = True
                break
        if bad:
            continue
        out[k, 0] = lo
        out[k, 1] = hi
        k += 1
    return out


def point_box_distance(p: np.ndarray, boxes: np.ndarray) -> np.ndarray:
    """Euclidean distance from points p [m,3] to each box [b,2,3]; negative-free (0 inside).

    Returns [m, b].  Also used to detect points inside boxes (distance 0).
    """
    lo = boxes[None, :, 0, :]
    hi = boxes[None, :, 1, :]
    q = p[:, None, :]
    d = np.maximum(np.maximum(lo - q, q - hi), 0.0)
    return np.sqrt((d * d).sum(-1))


def inside_any_box(p: np.ndarray, boxes: np.ndarray, margin: float, grid: int = 32) -> np.ndarray:
    """True where p lies inside a box or within `margin` of its surface.

    Boxes are binned into a grid x grid x grid lattice over the unit cube so each
    point is tested only against the boxes overlapping its lattice cell.
    """
    n = p.shape[0]
    out = np.zeros(n, bool)
    if boxes.shape[0] == 0 or n == 0:
        return out
    lo = np.clip(np.floor((boxes[:, 0, :] - margin) * grid), 0, grid - 1).astype(np.int64)
    hi = np.clip(np.floor((boxes[:, 1, :] + margin) * grid), 0, grid - 1).astype(np.int64)
    cell_boxes = {}
    for b in range(boxes.shape[0]):
        for ix in range(lo[b, 0], hi[b, 0] + 1):
            for iy in range(lo[b, 1], hi[b, 1] + 1):
                for iz in range(lo[b, 2], hi[b, 2] + 1):
                    cell_boxes.setdefault((ix * grid + iy) * grid + iz, []).append(b)
    pc = np.clip(np.floor(p * grid), 0, grid - 1).astype(np.int64)
    cid = (pc[:, 0] * grid + pc[:, 1]) * grid + pc[:, 2]
    order = np.argsort(cid, kind="stable")
    sc = cid[order]
    starts = np.flatnonzero(np.r_[True, sc[1:] != sc[:-1]])
    ends = np.r_[starts[1:], n]
    for s, e in zip(starts, ends):
        bl = cell_boxes.get(int(sc[s]))
        if not bl:
            continue
        idx = order[s:e]
        out[idx] = (point_box_distance(p[idx], boxes[bl]) < margin).any(axis=1)
    return out


def icosphere(center, radius: float, subdiv: int) -> np.ndarray:
    """Triangulated sphere (20 * 4^subdiv triangles), outward winding, float32 [n,3,3]."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    vv = np.array(v) * radius + np.asarray(center, np.float64)
    return vv[np.array(f)].astype(np.float32)
