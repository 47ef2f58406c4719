"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package holds none of the radiance-caching arithmetic: it only draws scenes
(triangle soups with per-triangle albedo), medium and light settings, record
positions and query points from seeded generators.  Every array it returns is
float32 (or int), so the CUDA library and the FP64 oracle read bit-identical
inputs (the oracle widens each float32 exactly to float64).

The scenes stand in for the paper's box-and-wall scenes (Sec. 6: Statues,
Patio, Strips, Cornell Holes, ...), which are not available: homogeneous media
in the unit cube, Lambertian boxes and walls, one point light, ray-march step
0.1 (Sec. 6, "Results in 3D").
"""
from .scenes import Scene, Medium, PointLight, box_triangles, cube_walls, ground_quads
from .configs import (RecordParams, Workload, config1, config2, config3, config4, config5,
                      get_config, record_positions, query_points, band_counts_loguniform)

__all__ = [
    "Scene", "Medium", "PointLight", "box_triangles", "cube_walls", "ground_quads",
    "RecordParams", "Workload", "config1", "config2", "config3", "config4", "config5",
    "get_config", "record_positions", "query_points", "band_counts_loguniform",
]
