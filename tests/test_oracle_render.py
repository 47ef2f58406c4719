"""Pins of the render oracle (oracle/render.py, CPU): the pinhole camera, the cube span and
the ray-march weights of Sec. 6's uniform marching, each against what geometry and the
closed-form integral fix."""
import math

import numpy as np

import oracle as O
import oracle.render as R
from workloads.scenes import Medium, PointLight, Scene


def test_camera_axes_and_field_of_view():
    W, H = 1920, 1080
    cam = R.camera((0.5, -0.8, 0.5), (0.0, 1.0, 0.0), 45.0, W, H)
    assert np.allclose(cam["r"], [1, 0, 0]) and np.allclose(cam["u"], [0, 0, 1])
    # the four central pixels are symmetric about the forward axis
    d = R.pixel_dirs(cam, [W // 2 - 1, W // 2, W // 2 - 1, W // 2], [H // 2 - 1, H // 2 - 1, H // 2, H // 2])
    assert np.allclose(d.mean(0) / np.linalg.norm(d.mean(0)), [0, 1, 0], atol=1e-12)
    # the top row's centres sit half a pixel inside the vertical half-angle
    top = R.pixel_dirs(cam, [W // 2], [0])[0]
    half = math.atan2(top[2], top[1])
    want = math.atan((1.0 - 1.0 / H) * math.tan(math.radians(22.5)))
    assert abs(half - want) < 1e-12
    # horizontal extent scales with the aspect ratio
    left = R.pixel_dirs(cam, [0], [H // 2])[0]
    assert abs(-left[0] / left[1] - (1.0 - 1.0 / W) * math.tan(math.radians(22.5)) * W / H) < 1e-3


def test_cube_span_on_the_faces():
    rng = np.random.default_rng(3)
    o = np.array([0.5, -0.8, 0.5])
    d = rng.normal(size=(500, 3)) * [0.3, 1.0, 0.3] + [0, 1.5, 0]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s_in, s_out, ok = R.cube_span(o, d)
    assert ok.any() and (~ok).any()
    for s in (s_in[ok], s_out[ok]):
        p = o + d[ok] * s[:, None]
        on_face = np.min(np.minimum(np.abs(p), np.abs(p - 1)), axis=1)
        assert np.all(on_face < 1e-12) and np.all((p > -1e-12) & (p < 1 + 1e-12))
    mid = o + d[ok] * (0.5 * (s_in[ok] + s_out[ok]))[:, None]
    assert np.all((mid > 0) & (mid < 1))
    inside = np.array([0.3, 0.4, 0.5])
    s_in, s_out, ok = R.cube_span(inside, d[:5])
    assert np.all(s_in == 0.0) and np.all(ok)


def test_march_weights_and_first_hit():
    """Midpoint weights sum to the closed form sigma_s (1 - e^(-sigma_t len)) / sigma_t within
    the midpoint rule's error, and the march ends at the first surface hit."""
    wall = np.array([[[0.0, 0.6, 0.0], [1.0, 0.6, 0.0], [1.0, 0.6, 1.0]],
                     [[0.0, 0.6, 0.0], [1.0, 0.6, 1.0], [0.0, 0.6, 1.0]]], np.float32)
    sc = Scene(tris=wall, albedo=np.full((2, 3), 0.7, np.float32), medium=Medium(0.4, 0.1, 0.7),
               lights=[PointLight((0.5, 0.5, 0.9), (1, 1, 1))])
    cam = R.camera((0.5, -0.8, 0.5), (0.0, 1.0, 0.0), 45.0, 64, 36)
    osc = O.OracleScene(sc, use_bvh=False)
    px, py = np.array([20, 32, 44]), np.array([10, 18, 25])
    steps = 64
    pts, wts, ok = R.march(osc, sc, cam, px, py, steps)
    assert np.all(ok)
    d = R.pixel_dirs(cam, px, py)
    s_in, _, _ = R.cube_span(cam["pos"], d)
    length = (0.6 - (cam["pos"][1] + d[:, 1] * s_in)) / d[:, 1]      # entry to the wall y = 0.6
    assert np.allclose(pts[:, -1, 1], cam["pos"][1] + d[:, 1] * (s_in + length * (steps - 0.5) / steps))
    sig_s, sig_t = float(np.float32(0.4)), float(np.float32(0.4) + np.float32(0.1))
    exact = sig_s * (1.0 - np.exp(-sig_t * length)) / sig_t
    ds = length / steps
    assert np.all(np.abs(wts.sum(1) - exact) <= sig_s * sig_t ** 2 * length * ds ** 2 / 24 * 1.01 + 1e-15)


def test_stored_crop_pixels_are_the_oracles():
    """The stored FP64 crop (oracle/render_crop_64.npz, written by `python -m oracle.render`)
    holds the oracle's own pixels: two of them recomputed here, with the record ids the crop
    gives their march points, match to rounding."""
    import os

    import workloads as W
    path = R.render_crop_pixels_path(64)
    assert os.path.exists(path)
    z = np.load(path)
    w = W.config5()
    ex = w.extra
    cam = R.camera(ex["camera"], ex["forward"], ex["vfov_deg"], ex["width"], ex["height"])
    size, steps = int(z["w"]), int(z["steps"])
    assert (int(z["x0"]), int(z["y0"])) == ((ex["width"] - size) // 2, (ex["height"] - size) // 2)
    for cx, cy in ((5, 9), (40, 62)):
        r0 = cy - cy % 4                     # the crop is computed in blocks of 4 pixel rows
        base = r0 * size * steps + ((cy - r0) * size + cx) * steps
        one = R.crop(w.scene, w.params, cam, int(z["x0"]) + cx, int(z["y0"]) + cy, 1, 1, steps, rec_base=base)
        assert np.allclose(one["img"][0, 0], z["img"][cy, cx], rtol=1e-12, atol=1e-15)
