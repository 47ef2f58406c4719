"""FP64 oracle of the render-shaped workload's pixels (test infrastructure only).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's measurement legs may import this
module; the product library never does.  It restates, in double precision, the paper's
rendering by uniform ray marching through the medium (Sec. 6): a pinhole camera's ray
enters the unit cube at s_in, is marched to the first surface hit or the cube exit in
`steps` equal segments, and a pixel is the sum over the segment midpoints x_k of
ds sigma_s exp(-sigma_t (s_k - s_in)) L(x_k).  Here L(x_k) is a full oracle record at every
march point (no cache, no interpolation): the reference the cached renderings are measured
against.  Camera: forward axis f, right = f x (0, 0, 1) normalised, up = right x f, vertical
field of view vfov; pixel (px, py) looks along f + right x + up y with
x = (2 (px + 1/2) / W - 1) tan(vfov / 2) W / H and y = (1 - 2 (py + 1/2) / H) tan(vfov / 2).

Usage (computes and caches the central crop of the render workload):
    python -m oracle.render [--size 64] [--threads N] [--out PATH]
Besides the full cache (per-march-point radiance, in the git-ignored cache directory) it writes
the composited pixels alone next to this file (render_crop_<size>.npz): the expected image that
the benchmark's equal-error comparison reads when the cache is absent.
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import OracleScene, records, trace

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def camera(pos, forward, vfov_deg: float, W: int, H: int) -> dict:
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, [0.0, 0.0, 1.0])
    if np.linalg.norm(r) < 1e-6:
        r = np.array([1.0, 0.0, 0.0])
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    return dict(pos=np.asarray(pos, np.float64), f=f, r=r, u=u, tan_half=math.tan(math.radians(0.5 * vfov_deg)),
                aspect=W / H, W=W, H=H)


def pixel_dirs(cam: dict, px, py) -> np.ndarray:
    px, py = np.asarray(px, np.float64), np.asarray(py, np.float64)
    x = (2.0 * (px + 0.5) / cam["W"] - 1.0) * cam["tan_half"] * cam["aspect"]
    y = (1.0 - 2.0 * (py + 0.5) / cam["H"]) * cam["tan_half"]
    d = cam["f"][None] + cam["r"][None] * x[:, None] + cam["u"][None] * y[:, None]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def cube_span(o, d):
    """Entry and exit parameters of rays o + s d in the unit cube (slab method)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        a = (0.0 - o[None]) / d
        b = (1.0 - o[None]) / d
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    lo = np.where(d == 0.0, -np.inf, lo)
    hi = np.where(d == 0.0, np.inf, hi)
    s_in = np.maximum(lo.max(axis=1), 0.0)
    s_out = hi.min(axis=1)
    return s_in, s_out, s_out > s_in


def march(oscene: OracleScene, scene, cam: dict, px, py, steps: int):
    """March points [n_pix, steps, 3], their pixel weights ds sigma_s exp(-sigma_t s_k)
    [n_pix, steps] and the valid-pixel mask."""
    d = pixel_dirs(cam, px, py)
    o = cam["pos"]
    s_in, s_out, ok = cube_span(o, d)
    e = o[None] + d * s_in[:, None]
    ids, t, _, _ = trace(oscene, e, d)
    length = np.where((ids >= 0) & (t < s_out - s_in + 1e-4), t, s_out - s_in)
    ok = ok & (length > 0)
    ds = length / steps
    s = (np.arange(steps)[None] + 0.5) * ds[:, None]
    pts = o[None, None] + d[:, None] * (s_in[:, None] + s)[..., None]
    sig_s = float(np.float32(scene.medium.sigma_s))
    sig_t = float(np.float32(scene.medium.sigma_t))
    wts = ds[:, None] * sig_s * np.exp(-sig_t * s)
    wts[~ok] = 0.0
    return pts, wts, ok


def crop(scene, params, cam: dict, x0: int, y0: int, w: int, h: int, steps: int, n_threads: int = 0,
         track_margins: int = 0, rec_base: int = 0) -> dict:
    """The FP64 reference of the pixels [x0, x0 + w) x [y0, y0 + h): a full oracle record
    (params; record ids = rec_base + march point index, march points in pixel-row order, `steps`
    per pixel) at every march point, composited.  With
    track_margins, img_budget bounds the change of each pixel that the records' near-tie
    decisions can make (their radiance budgets, weighted as the pixel sums them)."""
    osc = OracleScene(scene)
    py, px = np.mgrid[y0:y0 + h, x0:x0 + w]
    pts, wts, ok = march(osc, scene, cam, px.ravel(), py.ravel(), steps)
    flat = pts.reshape(-1, 3)
    L = np.zeros((flat.shape[0], 3))
    bud = np.zeros((flat.shape[0], 3))
    sel = np.repeat(ok, steps)
    ids = np.flatnonzero(sel)
    if ids.size:
        r = records(osc, params, flat[ids], rec_ids=rec_base + ids, n_threads=n_threads, track_margins=track_margins)
        L[ids] = r["L"]
        bud[ids] = r["bud_L"]
    img = (wts[..., None] * L.reshape(-1, steps, 3)).sum(axis=1)
    out = dict(img=img.reshape(h, w, 3), L=L.reshape(h, w, steps, 3).astype(np.float32), valid=ok.reshape(h, w),
               x0=x0, y0=y0, w=w, h=h, steps=steps)
    if track_margins:
        out["img_budget"] = (wts[..., None] * bud.reshape(-1, steps, 3)).sum(axis=1).reshape(h, w, 3)
        out["pts"] = pts.reshape(h, w, steps, 3)
    return out


def render_crop_path(size: int = 64) -> str:
    return os.path.join(CACHE_DIR, f"render_crop_{size}.npz")


def render_crop_pixels_path(size: int = 64) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"render_crop_{size}.npz")


PIXEL_KEYS = ("img", "valid", "x0", "y0", "w", "h", "steps", "seconds")


def crop_available(size: int = 64) -> bool:
    return os.path.exists(render_crop_path(size)) or os.path.exists(render_crop_pixels_path(size))


def central_crop(size: int = 64, n_threads: int = 0, out: str = None, verbose: bool = False) -> dict:
    """The render workload's central size x size pixels (cached); record ids are the march
    points' indices over the whole crop (pixel rows in order, `steps` points per pixel)."""
    import workloads as W
    w = W.config5()
    ex = w.extra
    path = out or render_crop_path(size)
    for p in (path, render_crop_pixels_path(size)):
        if os.path.exists(p):
            z = np.load(p)
            return {k: z[k] for k in z.files}
    cam = camera(ex["camera"], ex["forward"], ex["vfov_deg"], ex["width"], ex["height"])
    x0, y0 = (ex["width"] - size) // 2, (ex["height"] - size) // 2
    t0 = time.time()
    # in blocks of rows, each kept on disk as it completes, so an interrupted run resumes
    rows, parts = 4, []
    for r0 in range(0, size, rows):
        part = path + f".rows{r0}.npz"
        if not os.path.exists(part):
            p = crop(w.scene, w.params, cam, x0, y0 + r0, size, min(rows, size - r0), ex["steps"], n_threads,
                     rec_base=r0 * size * ex["steps"])
            os.makedirs(os.path.dirname(path), exist_ok=True)
            np.savez(part + ".tmp.npz", **p)
            os.replace(part + ".tmp.npz", part)
            if verbose:
                print(f"rows {r0}..{r0 + rows}: {time.time() - t0:.0f} s", flush=True)
        z = np.load(part)
        parts.append({k: z[k] for k in ("img", "L", "valid")})
    res = {k: np.concatenate([q[k] for q in parts], axis=0) for k in ("img", "L", "valid")}
    res.update(x0=x0, y0=y0, w=size, h=size, steps=ex["steps"])
    res["seconds"] = time.time() - t0
    if verbose:
        print(f"crop {size}x{size}x{ex['steps']}: {res['seconds']:.0f} s")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path + ".tmp.npz", **res)
    os.replace(path + ".tmp.npz", path)
    write_pixels(res, render_crop_pixels_path(size))
    for r0 in range(0, size, rows):
        os.remove(path + f".rows{r0}.npz")
    return res


def write_pixels(res: dict, path: str) -> None:
    """The composited crop alone (the pixels, their mask and the crop's placement)."""
    np.savez_compressed(path + ".tmp.npz", **{k: np.asarray(res[k]) for k in PIXEL_KEYS})
    os.replace(path + ".tmp.npz", path)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=64)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--pixels-only", action="store_true",
                    help="rewrite the pixel file from an existing full cache, without recomputing")
    a = ap.parse_args()
    if a.pixels_only:
        z = np.load(a.out or render_crop_path(a.size))
        write_pixels({k: z[k] for k in z.files}, render_crop_pixels_path(a.size))
    else:
        central_crop(a.size, a.threads, a.out, verbose=True)
