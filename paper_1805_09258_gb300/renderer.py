"""A frame of the render-shaped workload (Sec. 6): pre-populate the cache from a strided
subset of camera rays, render every pixel from the cache, then add records for the
pixels whose march points no record covered and render those pixels again, until none
is left (the paper adds a record wherever a render-time look-up finds no valid record).

Only library calls: vrc_march_points / vrc_march_pixels, the placement waves
(placement.place), vrc_render / vrc_render_pixels, vrc_compact_indices.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import Camera, Scene, _torch, compact_indices, march_pixels, march_points, render, render_pixels
from .placement import place


@dataclass
class FrameResult:
    image: object
    seconds: float
    n_records: int
    passes: list = field(default_factory=list)
    misses: int = 0
    placement: object = None


def render_frame(scene: Scene, cam: Camera, params, steps: int = 64, stride: int = 4, mlp=None, coarse_params=None,
                 cell_over_radius: float = 1.5, start_level: int = 2, max_level: int = 7, max_repairs: int = 8,
                 aniso: bool = False):
    torch = _torch()
    W, H = cam.width, cam.height
    t0 = time.perf_counter()
    w, h = (W + stride - 1) // stride, (H + stride - 1) // stride
    pts, valid = march_points(scene, cam, 0, 0, w, h, stride, steps)
    pl = place(scene, params, pts, start_level, max_level, mlp, coarse_params, cell_over_radius, valid=valid,
               aniso=aniso)
    passes = [("prepass", int(pts.shape[0]), pl.n_records)]
    img = torch.empty((W * H, 3), dtype=torch.float32, device="cuda")
    miss = torch.empty((W * H,), dtype=torch.int32, device="cuda")
    render(scene, pl.grid, cam, 0, 0, W, H, steps, img, miss)
    scratch = torch.empty((2 * W * H + W * H // 1024 + 2,), dtype=torch.int32, device="cuda")
    pix = torch.empty((W * H,), dtype=torch.int32, device="cuda")
    misses = 0
    for _ in range(max_repairs):
        m = compact_indices(miss, scratch, pix)
        if m == 0:
            break
        misses += m
        plist = pix[:m].contiguous()
        mpts, mvalid = march_pixels(scene, cam, plist, steps)
        before = pl.n_records
        pl = place(scene, params, mpts, max_level, max_level, None, None, cell_over_radius, valid=mvalid, base=pl,
                   capacity=pl.n_records + int(mpts.shape[0]), aniso=aniso)
        passes.append(("repair", m, pl.n_records - before))
        render_pixels(scene, pl.grid, cam, plist, steps, img, miss)
    torch.cuda.synchronize()
    return FrameResult(image=img, seconds=time.perf_counter() - t0, n_records=pl.n_records, passes=passes,
                       misses=misses, placement=pl)
