"""FP64 CPU oracle for second-order occlusion-aware volumetric radiance caching.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the product library never does.  The
oracle is plain C (vrc_oracle.c, double precision, written for readability)
loaded through ctypes.  It shares no code with the CUDA library.

Every function in vrc_oracle.c cites the passage of the paper it follows
(Marco et al., "Second-Order Occlusion-Aware Volumetric Radiance Caching",
TOG 37(2), 2018): Sec. 3 Eqs. outLF/mediaLFin/curveLFin, Sec. 4
Eqs. ApprxRadiance .. reducedRadianceDerivatives, Sec. 5 Eqs. errorTaylor,
radiusAniso3D, radianceTaylor, App. A (transmittance), App. C (triangle form
factor), Sec. 6 "Implementation" (stratified sphere, shells by ray marching).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_vrc.so")
OUT_STRIDE = 132

# output slots (see the enum in vrc_oracle.c)
SLOTS = dict(L=(0, 3), L_ss=(3, 3), L_ms=(6, 3), grad=(9, 9), grad_ss=(18, 9), grad_ms=(27, 9),
             hess=(36, 18), hess_ss=(54, 18), hess_ms=(72, 18), L_ff=(90, 3), radius=(93, 1),
             eig=(94, 3), kappa=(97, 1), status=(98, 1), n_shells=(99, 1), margin_edge=(100, 1),
             margin_t=(101, 1), n_rays=(102, 1), n_degen=(103, 1), L_ff_ss=(104, 3),
             L_ff_ms=(107, 3), L_Y=(110, 1), lam_max=(111, 1), bud_L=(112, 3), bud_L_ff=(115, 3),
             bud_grad=(118, 3), bud_hess=(121, 3), n_prim_unc=(124, 1), n_unc=(125, 1), n_replayed=(126, 1),
             n_bad_replay=(127, 1), n_lit_replayed=(128, 1), n_unexplained=(129, 1))


def build(force: bool = False) -> str:
    """Compile vrc_oracle.c with gcc into liboracle_vrc.so (in place)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _SceneIn(C.Structure):
    _fields_ = [("n_tris", C.c_int), ("tri_v", C.c_void_p), ("albedo", C.c_void_p),
                ("emission", C.c_void_p), ("sigma_s", C.c_float), ("sigma_a", C.c_float),
                ("g", C.c_float), ("n_lights", C.c_int), ("light_pos", C.c_void_p),
                ("light_I", C.c_void_p), ("use_bvh", C.c_int), ("sphere_mode", C.c_int),
                ("sphere_c", C.c_float * 3), ("sphere_r", C.c_float), ("sphere_Le", C.c_float * 3)]


class _Params(C.Structure):
    _fields_ = [("n_bands", C.c_int), ("n_bins", C.c_int), ("dt", C.c_float), ("eps", C.c_float),
                ("omega_o", C.c_float * 3), ("seed", C.c_uint64), ("ff_signed", C.c_int),
                ("extrap_order", C.c_int), ("r_min", C.c_float), ("r_max", C.c_float),
                ("rec_base", C.c_int64), ("general_derivs", C.c_int), ("track_margins", C.c_int),
                ("surface_only", C.c_int), ("lo_grad", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_scene_create.restype = P
        _lib.orc_scene_create.argtypes = [P]
        _lib.orc_scene_destroy.argtypes = [P]
        _lib.orc_records.argtypes = [P, P, P, P, P, C.c_int, P, C.c_int, P, P, P, P, C.c_int, P, C.c_int,
                                     P, P, P, C.c_int, C.c_int]
        _lib.orc_frozen_eval.argtypes = [P, P, P, C.c_int64, P, C.c_int, C.c_int, P]
        _lib.orc_hg.restype = C.c_double
        _lib.orc_hg.argtypes = [C.c_double, C.c_double]
        _lib.orc_radius.restype = C.c_double
        _lib.orc_radius.argtypes = [C.c_double, P, C.c_double, C.c_double, C.c_double, P, P]
        _lib.orc_eig3.argtypes = [P, P]
        _lib.orc_ray_directions.argtypes = [P, C.c_int64, P]
        _lib.orc_jitter.restype = C.c_double
        _lib.orc_jitter.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_int, C.c_int]
        _lib.orc_splitmix64.restype = C.c_uint64
        _lib.orc_splitmix64.argtypes = [C.c_uint64]
        _lib.orc_formfactor.argtypes = [P, P, P, P, C.c_int, P]
        _lib.orc_transmittance.argtypes = [P, P, C.c_double, P]
        _lib.orc_phase.argtypes = [P, P, P, C.c_double, P]
        _lib.orc_cell.argtypes = [P, P, P, P, C.c_int, P, C.c_double, C.c_double, P, C.c_double,
                                  C.c_int, C.c_int, P]
        _lib.orc_cell_vertices.argtypes = [C.c_int, C.c_int, C.c_int, P]
        _lib.orc_trace.argtypes = [P, P, P, C.c_int, P, P, P, P]
        _lib.orc_query.argtypes = [P, P, P, P, P, C.c_int, P, C.c_int, C.c_int, P, P, P]
        _lib.orc_query_aniso.argtypes = [P, P, P, P, P, C.c_int, P, C.c_int, C.c_int, P, P, P]
        _lib.orc_aniso.argtypes = [C.c_double, P, C.c_double, C.c_double, C.c_double, P, P, P, P]
        _lib.orc_coarse_features.argtypes = [P, P, P, P, C.c_int, P, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class OracleScene:
    """A scene as the oracle sees it (triangles widened exactly from float32 to double)."""

    def __init__(self, scene=None, use_bvh: Optional[bool] = None, sphere=None):
        self._keep = []
        s = _SceneIn()
        if scene is not None:
            tris = _f32(scene.tris)
            alb = _f32(scene.albedo)
            em = None if scene.emission is None else _f32(scene.emission)
            lp, li = scene.light_arrays()
            lp, li = _f32(lp), _f32(li)
            self._keep += [tris, alb, em, lp, li]
            s.n_tris = tris.shape[0]
            s.tri_v, s.albedo, s.emission = _p(tris), _p(alb), _p(em)
            s.sigma_s, s.sigma_a, s.g = scene.medium.sigma_s, scene.medium.sigma_a, scene.medium.g
            s.n_lights = lp.shape[0]
            s.light_pos, s.light_I = _p(lp), _p(li)
            s.use_bvh = int(tris.shape[0] > 64 if use_bvh is None else use_bvh)
        if sphere is not None:
            # closed-form test mode: x inside a sphere of constant inward radiance,
            # pure absorber (sigma_s = 0), no lights
            s.sphere_mode = 1
            s.sphere_c[:] = list(sphere["center"])
            s.sphere_r = sphere["radius"]
            s.sphere_Le[:] = list(sphere["Le"])
            s.sigma_s, s.sigma_a, s.g = 0.0, sphere["sigma_t"], sphere.get("g", 0.0)
        self._in = s
        self.ptr = lib().orc_scene_create(C.byref(s))

    def __del__(self):
        try:
            if self.ptr:
                lib().orc_scene_destroy(self.ptr)
        except Exception:
            pass


def make_params(rp, general_derivs: int = 1, track_margins: int = 0, surface_only: int = 0) -> _Params:
    p = _Params()
    p.n_bands, p.n_bins = rp.n_bands, rp.n_bins
    p.dt, p.eps = rp.dt, rp.eps
    p.omega_o[:] = list(rp.omega_o)
    p.seed = rp.seed
    p.ff_signed, p.extrap_order = rp.ff_signed, rp.extrap_order
    p.r_min, p.r_max = rp.r_min, rp.r_max
    p.rec_base = rp.rec_base
    p.general_derivs, p.track_margins, p.surface_only = general_derivs, track_margins, surface_only
    p.lo_grad = int(getattr(rp, "lo_grad", 0))
    return p


def records(oscene: OracleScene, rp, pos, rec_ids=None, n_bands=None, n_threads: int = 0,
            debug: bool = False, general_derivs: int = 1, track_margins: int = 0,
            surface_only: int = 0, replay_hits=None, replay_t=None, replay_lit=None) -> dict:
    """Compute records at positions `pos` [n,3] (float32).  Returns named float64 arrays.

    Replay mode (the discrete decisions of a record taken as given, its arithmetic in FP64):
    replay_hits (int [n, S], S >= rays): a primary hit primitive id per ray (ray order,
    the two pole rays last, -1 = no hit) used instead of the oracle's own closest hit;
    no primary-ray decision then enters the decision budgets (`n_replayed` counts the rays
    whose id differed).  With replay_t (float32 [n, S], each ray's end as computed in FP32:
    it decides which shell vertices are clamped and which vertices of a cell are furthest)
    and replay_lit (uint32 [n, shells, ceil(S / 32)], bit v of row k set when vertex v of
    shell k has radiance: the visibility decisions) every decision is the given one and the
    budgets are zero; `n_lit_replayed` counts visibility decisions taken the given way (each
    a shadow ray near an edge here) and `n_unexplained` given decisions that are not near
    ties in FP64."""
    pos = _f32(pos).reshape(-1, 3)
    n = pos.shape[0]
    rh = rt = rl = None
    n_sh = 0
    if replay_hits is not None:
        rh = np.ascontiguousarray(replay_hits, dtype=np.int32).reshape(n, -1)
    if replay_t is not None or replay_lit is not None:
        assert rh is not None and replay_t is not None and replay_lit is not None
        rt = np.ascontiguousarray(replay_t, dtype=np.float32).reshape(n, rh.shape[1])
        rl = np.ascontiguousarray(replay_lit).view(np.uint32).reshape(n, -1, (rh.shape[1] + 31) // 32)
        n_sh = rl.shape[1]
    ids = None if rec_ids is None else np.ascontiguousarray(rec_ids, dtype=np.int64)
    nb = None if n_bands is None else np.ascontiguousarray(n_bands, dtype=np.int32)
    out = np.zeros((n, OUT_STRIDE), np.float64)
    p = make_params(rp, general_derivs, track_margins, surface_only)
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    stride = 0
    dh = dt = dm = dtie = dl = None
    dshells = 0
    if debug:
        stride = int((nb.max() * 2 * nb.max() + 2) if nb is not None else rp.n_bands * rp.n_bins + 2)
        dh = np.full((n, stride), -2, np.int32)
        dt, dm, dtie = (np.zeros((n, stride)) for _ in range(3))
        dshells = int(np.ceil(np.sqrt(3.0) / float(rp.dt))) + 2
        dl = np.zeros((n, dshells, (stride + 31) // 32), np.uint32)
    lib().orc_records(oscene.ptr, C.byref(p), _p(pos), _p(ids), _p(nb), n, _p(out), n_threads,
                      _p(dh), _p(dt), _p(dm), _p(dtie), stride, _p(dl), dshells, _p(rh), _p(rt), _p(rl),
                      0 if rh is None else rh.shape[1], n_sh)
    res = {k: out[:, a:a + w] if w > 1 else out[:, a] for k, (a, w) in SLOTS.items()}
    res["status"] = res["status"].astype(np.int32)
    res["n_shells"] = res["n_shells"].astype(np.int32)
    for k in ("n_replayed", "n_lit_replayed", "n_unexplained"):
        res[k] = res[k].astype(np.int32)
    if debug:
        res.update(hit_prim=dh, hit_t=dt, hit_margin=dm, hit_tie=dtie, lit=dl)
    return res


def frozen_eval(oscene: OracleScene, rp, x0, x_eval, rec: int = 0, which: int = 0,
                general_derivs: int = 1, surface_only: int = 0):
    """L_ff and its analytic derivatives at x_eval with the record at x0 frozen.

    which: 0 all shells, 1 surface shell only, 2 medium shells only.
    Returns (L [m,3], grad [m,3,3], hess [m,3,3,3]).
    """
    x_eval = _f64(x_eval).reshape(-1, 3)
    out = np.zeros((x_eval.shape[0], 39))
    p = make_params(rp, general_derivs, 0, surface_only)
    x0a = _f32(x0)
    lib().orc_frozen_eval(oscene.ptr, C.byref(p), _p(x0a), rec, _p(x_eval), x_eval.shape[0], which, _p(out))
    return out[:, :3], out[:, 3:12].reshape(-1, 3, 3), out[:, 12:].reshape(-1, 3, 3, 3)


def _unpack13(o):
    return o[0], o[1:4].copy(), o[4:].reshape(3, 3).copy()


def formfactor(x, y1, y2, y3, ff_signed: int = 1):
    """App. C: F = Omega/4pi, grad F, H F (full 3x3).  Returns (F, g, H, ok)."""
    a = [_f64(v) for v in (x, y1, y2, y3)]
    o = np.zeros(13)
    ok = lib().orc_formfactor(*[_p(v) for v in a], ff_signed, _p(o))
    return (*_unpack13(o), ok)


def transmittance(x, y, sigma_t: float):
    a = [_f64(v) for v in (x, y)]
    o = np.zeros(13)
    lib().orc_transmittance(_p(a[0]), _p(a[1]), sigma_t, _p(o))
    return _unpack13(o)


def phase(x, y, wo, g: float):
    a = [_f64(v) for v in (x, y, wo)]
    o = np.zeros(13)
    lib().orc_phase(_p(a[0]), _p(a[1]), _p(a[2]), g, _p(o))
    return _unpack13(o)


def hg(mu: float, g: float) -> float:
    return lib().orc_hg(mu, g)


def cell(x, y1, y2, y3, far, Lo, sigma_t, g, wo, weight=1.0, general=1, ff_signed=1):
    """One cell's L_j, grad L_j, H L_j (RGB).

    far: index (0..2) of the furthest vertex, or a list of tied furthest vertex indices.
    Lo: RGB radiance, either one triple for all vertices or a [3][3] array per vertex.
    """
    Lo = np.asarray(Lo, np.float64)
    Lo3 = np.ascontiguousarray(np.broadcast_to(Lo, (3, 3)) if Lo.ndim == 1 else Lo)
    mask = (1 << far) if np.isscalar(far) else sum(1 << int(q) for q in far)
    a = [_f64(v) for v in (x, y1, y2, y3, wo)]
    o = np.zeros(39)
    ok = lib().orc_cell(_p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), mask, _p(Lo3), sigma_t, g, _p(a[4]), weight,
                        general, ff_signed, _p(o))
    return o[:3], o[3:12].reshape(3, 3), o[12:].reshape(3, 3, 3), ok


def cell_vertices(nb: int, ns: int):
    out = np.zeros((2 * nb * ns, 3), np.int32)
    tmp = np.zeros(3, np.int32)
    for c in range(2 * nb * ns):
        lib().orc_cell_vertices(nb, ns, c, _p(tmp))
        out[c] = tmp
    return out


def eig3(h6) -> np.ndarray:
    h = _f64(h6)
    lam = np.zeros(3)
    lib().orc_eig3(_p(h), _p(lam))
    return lam


def radius(LY: float, h6, eps: float, r_min: float, r_max: float):
    h = _f64(h6)
    st = np.zeros(1, np.int32)
    lam = np.zeros(3)
    R = lib().orc_radius(LY, _p(h), eps, r_min, r_max, _p(st), _p(lam))
    return R, int(st[0]), lam


LUM = np.array([0.2126, 0.7152, 0.0722])     # Rec.709 luminance weights (R15)


def aniso(LY: float, h6, eps: float, r_min: float, r_max: float):
    """Ellipsoidal record region (R17): (lam[3] ascending, radii[3], axes[3,3] rows =
    unit eigenvectors, metric[6] upper triangle of M = sum v v^T / R^2, status bits)."""
    h = _f64(h6)
    lam, radii, axes, metric = np.zeros(3), np.zeros(3), np.zeros(9), np.zeros(6)
    st = lib().orc_aniso(LY, _p(h), eps, r_min, r_max, _p(lam), _p(radii), _p(axes), _p(metric))
    return lam, radii, axes.reshape(3, 3), metric, int(st)


def aniso_records(L, hess, eps: float, r_min: float, r_max: float):
    """aniso() for every record from its RGB radiance L [n,3] and Hessian hess [n,18]:
    the luminance L_Y = LUM . L and H_Y = sum_c LUM_c H_c.  Returns (radii [n,3],
    axes [n,3,3], metric [n,6], lam [n,3], status [n])."""
    L = np.asarray(L, np.float64).reshape(-1, 3)
    H = np.asarray(hess, np.float64).reshape(-1, 3, 6)
    n = L.shape[0]
    radii, axes, metric, lam = np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 6)), np.zeros((n, 3))
    status = np.zeros(n, np.int32)
    for k in range(n):
        LY = float(LUM[0] * L[k, 0] + LUM[1] * L[k, 1] + LUM[2] * L[k, 2])
        hY = LUM[0] * H[k, 0] + LUM[1] * H[k, 1] + LUM[2] * H[k, 2]
        lam[k], radii[k], axes[k], metric[k], status[k] = aniso(LY, hY, eps, r_min, r_max)
    return radii, axes, metric, lam, status


def metric_matrix(m6) -> np.ndarray:
    """[..., 6] upper triangles (xx xy xz yy yz zz) -> [..., 3, 3] symmetric matrices."""
    m6 = np.asarray(m6, np.float64)
    M = np.empty(m6.shape[:-1] + (3, 3))
    for e, (i, j) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        M[..., i, j] = m6[..., e]
        M[..., j, i] = m6[..., e]
    return M


def ray_directions(rp, rec: int = 0) -> np.ndarray:
    p = make_params(rp)
    out = np.zeros((rp.n_bands * rp.n_bins + 2, 3))
    lib().orc_ray_directions(C.byref(p), rec, _p(out))
    return out


def jitter(seed: int, rec: int, i: int, j: int, stream: int) -> float:
    return lib().orc_jitter(seed, rec, i, j, stream)


def splitmix64(x: int) -> int:
    return lib().orc_splitmix64(x)


def trace(oscene: OracleScene, o, d):
    o, d = _f64(o).reshape(-1, 3), _f64(d).reshape(-1, 3)
    n = o.shape[0]
    ids = np.zeros(n, np.int32)
    t, m, tie = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_trace(oscene.ptr, _p(o), _p(d), n, _p(ids), _p(t), _p(m), _p(tie))
    return ids, t, m, tie


def query(rec_pos, rec_R, rec_L, rec_grad, rec_hess, q, order: int = 1):
    """Eq. radianceTaylor by brute force over all records.  Returns (rgb, count, near)."""
    rec_pos, rec_R, rec_L, rec_grad = (_f64(a) for a in (rec_pos, rec_R, rec_L, rec_grad))
    rec_hess = _f64(rec_hess) if rec_hess is not None else np.zeros((rec_pos.shape[0], 18))
    q = _f64(q).reshape(-1, 3)
    nq = q.shape[0]
    out = np.zeros((nq, 3))
    st = np.zeros(nq, np.int32)
    near = np.zeros(nq, np.int32)
    lib().orc_query(_p(rec_pos), _p(rec_R), _p(rec_L), _p(rec_grad), _p(rec_hess), rec_pos.shape[0], _p(q),
                    nq, order, _p(out), _p(st), _p(near))
    return out, st, near


def query_aniso(rec_pos, rec_metric, rec_L, rec_grad, rec_hess, q, order: int = 1):
    """Eq. radianceTaylor over ellipsoidal records (R17) by brute force.  Returns
    (rgb, count, near)."""
    rec_pos, rec_metric, rec_L, rec_grad = (_f64(a) for a in (rec_pos, rec_metric, rec_L, rec_grad))
    rec_hess = _f64(rec_hess) if rec_hess is not None else np.zeros((rec_pos.shape[0], 18))
    q = _f64(q).reshape(-1, 3)
    nq = q.shape[0]
    out = np.zeros((nq, 3))
    st = np.zeros(nq, np.int32)
    near = np.zeros(nq, np.int32)
    lib().orc_query_aniso(_p(rec_pos), _p(rec_metric), _p(rec_L), _p(rec_grad), _p(rec_hess), rec_pos.shape[0],
                          _p(q), nq, order, _p(out), _p(st), _p(near))
    return out, st, near


def coarse_features(oscene: OracleScene, rp, pos, rec_ids=None):
    """Features of the learned radius predictor for each position: log hit distance and
    to-light transmittance x visibility of the coarse ray set.  Returns (features [n, 2N],
    near-tie flags [n, 2N])."""
    pos = _f32(pos).reshape(-1, 3)
    n = pos.shape[0]
    N = rp.n_bands * rp.n_bins
    ids = None if rec_ids is None else np.ascontiguousarray(rec_ids, dtype=np.int64)
    out = np.zeros((n, 2 * N))
    unc = np.zeros((n, 2 * N), np.uint8)
    p = make_params(rp)
    lib().orc_coarse_features(oscene.ptr, C.byref(p), _p(pos), _p(ids), n, _p(out), _p(unc))
    return out, unc.astype(bool)
