"""The five seeded workloads (scene, medium, light, record and query sets).

| name | scene | records | rays per record | queries |
|------|-------|---------|-----------------|---------|
| small (config1) | cube walls + one box, 24 tris | 64 | 16 bands x 32 bins | 256 |
| mid (config2) | 170 random boxes + ground, 2,048 tris | 4,096 | 32 x 64 | 1M |
| batching (config3) | 8,333 boxes + ground, 100,000 tris | 100,000 | 8x16 .. 64x128 log-uniform | - |
| learned (config4) | 16 mid-style scenes | training set | 32 x 64 (+ coarse 8 x 16) | - |
| render (config5) | 170 tessellated boxes + ground grid, 250,040 tris | adaptive | 32 x 64 | 1920x1080x64 |

Common settings: medium fills the unit cube, one point light at (0.5, 0.5, 0.92)
with RGB intensity (1.0, 0.9, 0.8), Lambertian surfaces of albedo 0.7, march
step 0.1 (the paper's render step, Sec. 6), error tolerance 0.05, outgoing
direction +z.  Seeds: scene 1, records 2, ray jitter 3, queries 4.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

from .scenes import (Medium, PointLight, Scene, box_triangles, box_triangles_tessellated, cube_walls, ground_grid,
                     ground_quads, inside_any_box, random_boxes)

SEED_SCENE, SEED_RECORDS, SEED_JITTER, SEED_QUERIES = 1, 2, 3, 4
LIGHT_POS = (0.5, 0.5, 0.92)
LIGHT_I = (1.0, 0.9, 0.8)
SURFACE_ALBEDO = 0.7
POS_MARGIN = 1e-3


@dataclass
class RecordParams:
    """Per-call record parameters (mirrors the C struct vrc_record_params)."""
    n_bands: int = 16
    n_bins: int = 32
    dt: float = 0.1
    eps: float = 0.05
    omega_o: tuple = (0.0, 0.0, 1.0)
    seed: int = SEED_JITTER
    ff_signed: int = 1
    extrap_order: int = 1
    r_min: float = 1e-3
    r_max: float = 0.5
    rec_base: int = 0
    parts: int = 0          # 0 whole radiance, 1 surface shell (SS cache), 2 medium shells (MS cache)
    lo_grad: int = 0        # 1: medium vertices' radiance varies with x through their phase function

    @property
    def n_rays(self) -> int:
        return self.n_bands * self.n_bins + 2


@dataclass
class Workload:
    name: str
    scene: Scene
    params: RecordParams
    n_records: int
    n_queries: int
    band_counts: Optional[np.ndarray] = None      # per-record n_bands (batching workload)
    extra: dict = field(default_factory=dict)

    def positions(self, n: Optional[int] = None, seed: int = SEED_RECORDS) -> np.ndarray:
        return record_positions(self.scene, self.n_records if n is None else n, seed)

    def queries(self, n: Optional[int] = None, seed: int = SEED_QUERIES) -> np.ndarray:
        return query_points(self.scene, self.n_queries if n is None else n, seed)


def _uniform_outside_boxes(scene: Scene, n: int, seed: int, margin: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.zeros((0, 3), np.float32)
    while out.shape[0] < n:
        m = max(1024, int((n - out.shape[0]) * 1.3))
        p = rng.uniform(margin, 1.0 - margin, size=(m, 3)).astype(np.float32)
        keep = ~inside_any_box(p.astype(np.float64), scene.boxes.astype(np.float64), margin)
        out = np.concatenate([out, p[keep]], axis=0)
    return np.ascontiguousarray(out[:n])


def record_positions(scene: Scene, n: int, seed: int = SEED_RECORDS) -> np.ndarray:
    """Record centres: uniform in the cube, rejected inside boxes or within 1e-3 of a surface."""
    return _uniform_outside_boxes(scene, n, seed, POS_MARGIN)


def query_points(scene: Scene, n: int, seed: int = SEED_QUERIES) -> np.ndarray:
    """Query points: uniform in the cube, rejected inside boxes."""
    return _uniform_outside_boxes(scene, n, seed, POS_MARGIN)


def band_counts_loguniform(n: int, seed: int = SEED_RECORDS + 100) -> np.ndarray:
    """Per-record band counts N_b = round(8 * 2^(3u)), u ~ U[0,1): 8..64 bands, bins = 2 N_b."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=n)
    return np.clip(np.rint(8.0 * 2.0 ** (3.0 * u)), 8, 64).astype(np.int32)


def _box_scene(name: str, n_boxes: int, side_lo: float, side_hi: float, log_uniform: bool,
               n_ground: int, medium: Medium, seed: int) -> Scene:
    rng = np.random.default_rng(seed)
    boxes = random_boxes(rng, n_boxes, side_lo, side_hi, log_uniform,
                         keep_clear=[np.array(LIGHT_POS, np.float64)], clear_radius=0.02)
    tris = [box_triangles(b[0], b[1]) for b in boxes]
    tris.append(ground_quads(n_ground))
    tris = np.concatenate(tris, axis=0).astype(np.float32)
    albedo = np.full((tris.shape[0], 3), SURFACE_ALBEDO, np.float32)
    return Scene(tris=np.ascontiguousarray(tris), albedo=albedo, medium=medium,
                 lights=[PointLight(LIGHT_POS, LIGHT_I)], boxes=boxes, name=name)


def config1() -> Workload:
    """Small plain workload: 12 wall triangles + one centred box, 64 records at 16 x 32."""
    box = np.array([[[0.35, 0.35, 0.30], [0.65, 0.65, 0.60]]], np.float32)
    tris = np.concatenate([cube_walls(), box_triangles(box[0, 0], box[0, 1])], axis=0)
    scene = Scene(tris=np.ascontiguousarray(tris, dtype=np.float32),
                  albedo=np.full((tris.shape[0], 3), SURFACE_ALBEDO, np.float32),
                  medium=Medium(0.5, 0.05, 0.3), lights=[PointLight(LIGHT_POS, LIGHT_I)],
                  boxes=box, name="walls+box (24 tris)")
    return Workload("small: 24 tris, 64 records x 16x32 rays, 256 queries", scene,
                    RecordParams(n_bands=16, n_bins=32), n_records=64, n_queries=256)


def config2() -> Workload:
    """Mid plain workload: 2,048 triangles, 4,096 records at 32 x 64, 1M queries."""
    scene = _box_scene("170 boxes + ground (2,048 tris)", 170, 0.02, 0.2, False, 8,
                       Medium(0.8, 0.2, 0.5), SEED_SCENE)
    return Workload("mid: 2,048 tris, 4,096 records x 32x64 rays, 1M queries", scene,
                    RecordParams(n_bands=32, n_bins=64), n_records=4096, n_queries=1 << 20)


def config3() -> Workload:
    """Batching workload: 100,000 triangles, 100,000 records with 8x16 .. 64x128 rays.

    Box sides are log-uniform in [0.005, 0.025]: the boxes' optical depth is about 2.3 per
    unit length, so a shadow ray to the light is blocked with a probability well below
    one (sides of 0.01 .. 0.05 would give about 8 per unit length and an almost unlit
    scene, where every record's radius collapses to r_min)."""
    scene = _box_scene("8,333 boxes + ground (100,000 tris)", 8333, 0.005, 0.025, True, 4,
                       Medium(0.8, 0.2, 0.5), SEED_SCENE)
    n = 100_000
    return Workload("batching: 100k tris, 100k records, 8x16..64x128 rays", scene,
                    RecordParams(n_bands=64, n_bins=128), n_records=n, n_queries=0,
                    band_counts=band_counts_loguniform(n))


def config4(scene_seed: int = SEED_SCENE) -> Workload:
    """Learned-radius workload: mid-style scenes, full records at 32 x 64, coarse 8 x 16 features."""
    scene = _box_scene(f"170 boxes + ground, seed {scene_seed}", 170, 0.02, 0.2, False, 8,
                       Medium(0.8, 0.2, 0.5), scene_seed)
    return Workload("learned: mid-style scenes, 32x64 full / 8x16 coarse", scene,
                    RecordParams(n_bands=32, n_bins=64), n_records=4096, n_queries=0,
                    extra={"coarse": RecordParams(n_bands=8, n_bins=16, seed=SEED_JITTER + 1000)})


def render_scene(seed: int = SEED_SCENE) -> Scene:
    """170 boxes with sides U[0.02, 0.2] (the mid scene's distribution), every face
    tessellated into 11 x 11 quads, plus a 40 x 40 ground grid: 250,040 triangles.
    Boxes of this size cast shadows that a 32 x 64-ray record resolves; a field of
    thousands of millimetre boxes (tried first) gives radiance whose shadow structure is
    finer than the record's ray set, so no tolerance changes the frame's error."""
    rng = np.random.default_rng(seed)
    boxes = random_boxes(rng, 170, 0.02, 0.2, False, keep_clear=[np.array(LIGHT_POS, np.float64)],
                         clear_radius=0.02)
    tris = np.concatenate([box_triangles_tessellated(b[0], b[1], 11) for b in boxes] + [ground_grid(40)])
    tris = np.ascontiguousarray(tris, dtype=np.float32)
    albedo = np.full((tris.shape[0], 3), SURFACE_ALBEDO, np.float32)
    return Scene(tris=tris, albedo=albedo, medium=Medium(0.4, 0.1, 0.7), lights=[PointLight(LIGHT_POS, LIGHT_I)],
                 boxes=boxes, name="170 tessellated boxes + ground grid (250,040 tris)")


def config5() -> Workload:
    """Render-shaped workload: 250,040 triangles, 1920x1080 camera, 64 march steps."""
    scene = render_scene()
    return Workload("render: 250k tris, 1920x1080x64 march points", scene,
                    RecordParams(n_bands=32, n_bins=64, omega_o=(0.0, -1.0, 0.0)),
                    n_records=0, n_queries=1920 * 1080 * 64,
                    extra={"camera": (0.5, -0.8, 0.5), "forward": (0.0, 1.0, 0.0), "vfov_deg": 45.0,
                           "width": 1920, "height": 1080, "steps": 64})


def get_config(i: int) -> Workload:
    return {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}[i]()


def with_params(w: Workload, **kw) -> Workload:
    return replace(w, params=replace(w.params, **kw))
