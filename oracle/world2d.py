"""FP64 CPU oracle of the paper's two-dimensional world (vrc2d_oracle.c through ctypes).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU baseline
leg may import this module; the product library never does.  vrc2d_oracle.c cites the
passages it follows (Sec. 3 in 2D, Sec. 4, App. A, App. B, Eq. radiusAniso2D) and lists
its readings D1..D9.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrc2d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_vrc2d.so")
STRIDE = 72
SLOTS = dict(L=(0, 3), L_ss=(3, 3), L_ms=(6, 3), grad=(9, 6), grad_ss=(15, 6), grad_ms=(21, 6), hess=(27, 9),
             hess_ss=(36, 9), hess_ms=(45, 9), L_ff=(54, 3), radius=(57, 1), eig=(58, 2), status=(60, 1),
             n_shells=(61, 1), prim_near=(62, 1), bud_L=(63, 3), bud_grad=(66, 3), bud_hess=(69, 3))


def build(force: bool = False) -> str:
    """Compile vrc2d_oracle.c with gcc into liboracle_vrc2d.so (in place)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("n_segs", C.c_int), ("seg", C.c_void_p), ("albedo", C.c_void_p), ("sigma_s", C.c_float),
                ("sigma_a", C.c_float), ("n_lights", C.c_int), ("light_pos", C.c_void_p), ("light_I", C.c_void_p),
                ("circle_mode", C.c_int), ("circle_c", C.c_float * 2), ("circle_r", C.c_float),
                ("circle_Le", C.c_float * 3)]


class _Params(C.Structure):
    _fields_ = [("n_dirs", C.c_int), ("dt", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64),
                ("r_min", C.c_float), ("r_max", C.c_float), ("rec_base", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.o2_records.argtypes = [P, P, P, P, C.c_int, P, P, C.c_int]
        _lib.o2_frozen_eval.argtypes = [P, P, P, C.c_int64, P, P]
        _lib.o2_segment_angle.argtypes = [P, P, P, P]
        _lib.o2_transmittance.argtypes = [P, P, C.c_double, P]
        _lib.o2_ray_directions.argtypes = [P, C.c_int64, P]
        _lib.o2_trace.argtypes = [P, P, P, C.c_int, P, P]
        _lib.o2_radius.argtypes = [C.c_double, P, C.c_double, C.c_double, C.c_double, P, P]
        _lib.o2_radius.restype = C.c_double
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class OracleScene2:
    """A 2D scene (workloads.flat.Scene2) or the analytic constant-radiance circle."""

    def __init__(self, scene=None, circle=None, sigma_s=0.8, sigma_a=0.2):
        s = _Scene()
        self._keep = []
        if circle is not None:
            c, r, Le = circle
            s.n_segs = 0
            s.circle_mode = 1
            s.circle_c[:] = [float(c[0]), float(c[1])]
            s.circle_r = float(r)
            s.circle_Le[:] = [float(v) for v in Le]
            s.sigma_s, s.sigma_a = sigma_s, sigma_a
            s.n_lights = 0
        else:
            segs, alb = _f32(scene.segs), _f32(scene.albedo)
            lp, li = scene.light_arrays()
            lp, li = _f32(lp), _f32(li)
            self._keep += [segs, alb, lp, li]
            s.n_segs = segs.shape[0]
            s.seg, s.albedo = _p(segs), _p(alb)
            s.sigma_s, s.sigma_a = scene.sigma_s, scene.sigma_a
            s.n_lights = lp.shape[0]
            s.light_pos, s.light_I = _p(lp), _p(li)
            s.circle_mode = 0
        self.s = s

    @property
    def ptr(self):
        return C.byref(self.s)


def make_params(rp) -> _Params:
    p = _Params()
    p.n_dirs = int(rp.n_bins)
    p.dt, p.eps = float(rp.dt), float(rp.eps)
    p.seed = int(rp.seed)
    p.r_min, p.r_max = float(rp.r_min), float(rp.r_max)
    p.rec_base = int(getattr(rp, "rec_base", 0))
    return p


def records(oscene: OracleScene2, rp, pos, rec_ids=None, replay_hits=None) -> dict:
    """2D records at pos [n, 2] (float32).  Returns a dict of arrays keyed as SLOTS:
    grad [n, 3, 2], hess [n, 3, 3] (xx, xy, yy per channel).  replay_hits (int [n, >= N]):
    a primary hit segment id per ray (-1 = none) used instead of the oracle's own closest
    hit (replay mode); prim_near then counts no ray."""
    pos = _f32(pos).reshape(-1, 2)
    n = pos.shape[0]
    ids = None if rec_ids is None else np.ascontiguousarray(rec_ids, dtype=np.int64)
    rh = None if replay_hits is None else np.ascontiguousarray(replay_hits, dtype=np.int32).reshape(n, -1)
    out = np.zeros((n, STRIDE))
    p = make_params(rp)
    lib().o2_records(oscene.ptr, C.byref(p), _p(pos), _p(ids), n, _p(out), _p(rh), 0 if rh is None else rh.shape[1])
    res = {}
    for k, (o, w) in SLOTS.items():
        res[k] = out[:, o] if w == 1 else out[:, o:o + w]
    for k in ("grad", "grad_ss", "grad_ms"):
        res[k] = res[k].reshape(n, 3, 2)
    for k in ("hess", "hess_ss", "hess_ms"):
        res[k] = res[k].reshape(n, 3, 3)
    res["status"] = res["status"].astype(np.int32)
    return res


def frozen_eval(oscene: OracleScene2, rp, x0, rec: int, x_eval) -> dict:
    """The record built at x0 (ray set, shells, vertex radiance frozen) with its cells
    evaluated at x_eval: returns L_ff, grad, hess there."""
    out = np.zeros(STRIDE)
    p = make_params(rp)
    lib().o2_frozen_eval(oscene.ptr, C.byref(p), _p(_f32(x0)), rec, _p(_f64(x_eval)), _p(out))
    return dict(L_ff=out[54:57].copy(), grad=out[9:15].reshape(3, 2).copy(), hess=out[27:36].reshape(3, 3).copy())


def segment_angle(x, y0, y1):
    """App. B with the sign of D4: (theta, grad [2], hess [xx, xy, yy], ok)."""
    out = np.zeros(6)
    ok = lib().o2_segment_angle(_p(_f64(x)), _p(_f64(y0)), _p(_f64(y1)), _p(out))
    return out[0], out[1:3].copy(), out[3:6].copy(), bool(ok)


def transmittance(x, y, sigma_t):
    out = np.zeros(6)
    lib().o2_transmittance(_p(_f64(x)), _p(_f64(y)), sigma_t, _p(out))
    return out[0], out[1:3].copy(), out[3:6].copy()


def radius(LY, h3, eps, r_min, r_max):
    st = np.zeros(1, np.int32)
    lam = np.zeros(2)
    R = lib().o2_radius(LY, _p(_f64(h3)), eps, r_min, r_max, _p(st), _p(lam))
    return R, int(st[0]), lam


def ray_directions(rp, rec: int = 0) -> np.ndarray:
    p = make_params(rp)
    out = np.zeros((rp.n_bins, 2))
    lib().o2_ray_directions(C.byref(p), rec, _p(out))
    return out


def trace(oscene: OracleScene2, o, d):
    o, d = _f64(o).reshape(-1, 2), _f64(d).reshape(-1, 2)
    n = o.shape[0]
    ids = np.zeros(n, np.int32)
    t = np.zeros(n)
    lib().o2_trace(oscene.ptr, _p(o), _p(d), n, _p(ids), _p(t))
    return ids, t
