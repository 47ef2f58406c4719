"""Seeded inputs of the two-dimensional world (Sec. 3): line segments ("curves") in the
unit square, which a homogeneous medium fills, lit by point lights.  Like the rest of
this package it holds none of the method's arithmetic; every array is float32.

| name | scene | records | directions | queries |
|------|-------|---------|------------|---------|
| flat small | 4 walls + one rectangle occluder, 8 segments | 64 | 256 | 4,096 |
| flat mid | ground + 40 random rectangles, 161 segments | 4,096 | 512 | 1M |

Medium: sigma_s 0.8, sigma_a 0.2 (isotropic); curve albedo 0.7; one point light at
(0.5, 0.92) with RGB intensity (1.0, 0.9, 0.8); march step 0.1; tolerance 0.05.
2D records are stored as 3D records in the plane z = Z_PLANE (zero z components), so
the 3D record grid and query serve them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from .configs import RecordParams

Z_PLANE = 0.5
LIGHT_POS2 = (0.5, 0.92)
LIGHT_I2 = (1.0, 0.9, 0.8)
ALBEDO2 = 0.7


@dataclass
class Light2:
    pos: tuple
    intensity: tuple


@dataclass
class Scene2:
    segs: np.ndarray                 # float32 [n, 4]: x0 y0 x1 y1
    albedo: np.ndarray               # float32 [n, 3]
    sigma_s: float
    sigma_a: float
    lights: List[Light2]
    rects: np.ndarray = field(default_factory=lambda: np.zeros((0, 2, 2), np.float32))
    name: str = ""

    @property
    def n_segs(self) -> int:
        return int(self.segs.shape[0])

    def light_arrays(self):
        pos = np.array([l.pos for l in self.lights], np.float32).reshape(-1, 2)
        inten = np.array([l.intensity for l in self.lights], np.float32).reshape(-1, 3)
        return pos, inten


@dataclass
class Workload2:
    name: str
    scene: Scene2
    params: RecordParams             # n_bins = angular strata, n_bands = 1
    n_records: int
    n_queries: int

    def positions(self, n=None, seed: int = 2) -> np.ndarray:
        return points_outside(self.scene, self.n_records if n is None else n, seed)

    def queries(self, n=None, seed: int = 4) -> np.ndarray:
        return points_outside(self.scene, self.n_queries if n is None else n, seed)


def rect_segments(lo, hi) -> np.ndarray:
    (x0, y0), (x1, y1) = lo, hi
    return np.array([[x0, y0, x1, y0], [x1, y0, x1, y1], [x1, y1, x0, y1], [x0, y1, x0, y0]], np.float32)


def walls() -> np.ndarray:
    return rect_segments((0.0, 0.0), (1.0, 1.0))


def inside_rects(p: np.ndarray, rects: np.ndarray, margin: float) -> np.ndarray:
    out = np.zeros(p.shape[0], bool)
    for lo, hi in rects.astype(np.float64):
        out |= np.all((p >= lo - margin) & (p <= hi + margin), axis=1)
    return out


def points_outside(scene: Scene2, n: int, seed: int, margin: float = 1e-3) -> np.ndarray:
    """Uniform points of the square, rejected inside rectangles or within 1e-3 of one."""
    rng = np.random.default_rng(seed)
    out = np.zeros((0, 2), np.float32)
    while out.shape[0] < n:
        m = max(1024, int((n - out.shape[0]) * 1.3))
        p = rng.uniform(margin, 1.0 - margin, size=(m, 2)).astype(np.float32)
        keep = ~inside_rects(p.astype(np.float64), scene.rects, margin)
        out = np.concatenate([out, p[keep]], axis=0)
    return np.ascontiguousarray(out[:n])


def _scene(segs, rects, name):
    segs = np.ascontiguousarray(segs, np.float32)
    return Scene2(segs=segs, albedo=np.full((segs.shape[0], 3), ALBEDO2, np.float32), sigma_s=0.8, sigma_a=0.2,
                  lights=[Light2(LIGHT_POS2, LIGHT_I2)], rects=np.asarray(rects, np.float32).reshape(-1, 2, 2),
                  name=name)


def flat_small() -> Workload2:
    rect = np.array([[0.35, 0.35], [0.65, 0.6]], np.float32)
    segs = np.concatenate([walls(), rect_segments(rect[0], rect[1])])
    sc = _scene(segs, rect[None], "4 walls + rectangle (8 segments)")
    return Workload2("flat small: 8 segments, 64 records x 256 directions", sc,
                     RecordParams(n_bands=1, n_bins=256), n_records=64, n_queries=4096)


def random_rects(rng, n: int, side_lo: float, side_hi: float, clear=LIGHT_POS2, clear_r: float = 0.03):
    rects = []
    while len(rects) < n:
        c = rng.uniform(0, 1, 2)
        hs = 0.5 * rng.uniform(side_lo, side_hi, 2)
        lo, hi = np.clip(c - hs, 0, 1), np.clip(c + hs, 0, 1)
        if np.all(hi - lo > 1e-3) and not np.all(np.abs(np.asarray(clear) - np.clip(clear, lo, hi)) < clear_r):
            rects.append((lo, hi))
    return np.array(rects, np.float32)


def flat_mid() -> Workload2:
    rng = np.random.default_rng(1)
    rects = random_rects(rng, 40, 0.02, 0.12)
    ground = np.array([[0.0, 0.0, 1.0, 0.0]], np.float32)
    segs = np.concatenate([ground] + [rect_segments(lo, hi) for lo, hi in rects])
    sc = _scene(segs, rects, "ground + 40 rectangles (161 segments)")
    return Workload2("flat mid: 161 segments, 4,096 records x 512 directions", sc,
                     RecordParams(n_bands=1, n_bins=512), n_records=4096, n_queries=1 << 20)
