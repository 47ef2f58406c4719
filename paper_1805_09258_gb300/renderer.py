"""A frame of the render-shaped workload (Sec. 6): pre-populate the cache from a strided
subset of camera rays, render every pixel from the cache, then add records for the
pixels whose march points no record covered and render those pixels again, until none
is left (the paper adds a record wherever a render-time look-up finds no valid record).

With split=True the frame uses two caches, as Sec. 6 does: one of single-scattering
records (the surface shell alone, parts = 1) and one of multiple-scattering records (the
medium shells alone, parts = 2), each placed against its own radii; a march point's
radiance is the sum of both caches' look-ups.

Only library calls: vrc_march_points / vrc_march_pixels, the placement waves
(placement.place), vrc_render / vrc_render_pixels, vrc_compact_indices.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field, replace

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
    placement2: object = None      # the multiple-scattering cache when split
    placement_s: float = 0.0       # time in placement (records, grids, coverage), prepass and repairs


def render_frame(scene: Scene, cam: Camera, params, steps: int = 64, stride: int = 4, mlp=None, coarse_params=None,
                 cell_over_radius: float = 1.5, start_level: int = 2, max_level: int = 7, max_repairs: int = 8,
                 aniso: bool = False, split: bool = False, eps_train: float = None):
    torch = _torch()
    W, H = cam.width, cam.height
    t0 = time.perf_counter()
    w, h = (W + stride - 1) // stride, (H + stride - 1) // stride
    pts, valid = march_points(scene, cam, 0, 0, w, h, stride, steps)
    caches = [replace(params, parts=1), replace(params, parts=2)] if split else [params]
    pls = [place(scene, p, pts, start_level, max_level, mlp, coarse_params, cell_over_radius, valid=valid,
                 aniso=aniso, eps_train=eps_train) for p in caches]
    placement_s = sum(pl.seconds for pl in pls)
    passes = [("prepass", int(pts.shape[0]), sum(pl.n_records for pl in pls))]
    img = torch.empty((W * H, 3), dtype=torch.float32, device="cuda")
    miss = torch.empty((W * H,), dtype=torch.int32, device="cuda")

    def grid2():
        return pls[1].grid if split else None

    render(scene, pls[0].grid, cam, 0, 0, W, H, steps, img, miss, grid2=grid2())
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
        before = sum(pl.n_records for pl in pls)
        pls = [place(scene, p, mpts, max_level, max_level, None, None, cell_over_radius, valid=mvalid, base=pl,
                     capacity=pl.n_records + int(mpts.shape[0]), aniso=aniso) for p, pl in zip(caches, pls)]
        placement_s += sum(pl.seconds for pl in pls)
        passes.append(("repair", m, sum(pl.n_records for pl in pls) - before))
        render_pixels(scene, pls[0].grid, cam, plist, steps, img, miss, grid2=grid2())
    torch.cuda.synchronize()
    return FrameResult(image=img, seconds=time.perf_counter() - t0, n_records=sum(pl.n_records for pl in pls),
                       passes=passes, misses=misses, placement=pls[0], placement2=pls[1] if split else None,
                       placement_s=placement_s)
