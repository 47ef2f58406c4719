"""Python binding of libvrc (second-order occlusion-aware volumetric radiance caching).

Argument marshalling only: every step of the computation runs in the CUDA library
(libvrc.so, built from csrc/ for sm_103a).  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: if the library cannot be loaded or no
CUDA device is present, every call raises.

Names follow the C ABI in include/vrc.h: build_scene, compute_records,
compute_records_host, build_record_grid, query_inscatter.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvrc.so")

VRC_OK, VRC_ERR_INVALID, VRC_ERR_OOM, VRC_ERR_CUDA, VRC_ERR_TIMEOUT, VRC_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
REC_NONFINITE, REC_CLAMP_LO, REC_CLAMP_HI, REC_DEGENERATE = 1, 2, 4, 8
MAX_LIGHTS = 4


class VrcError(RuntimeError):
    pass


class _Medium(C.Structure):
    _fields_ = [("sigma_s", C.c_float), ("sigma_a", C.c_float), ("g", C.c_float)]


class _Light(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("intensity", C.c_float * 3)]


class RecordParamsC(C.Structure):
    _fields_ = [("n_bands", C.c_int32), ("n_bins", C.c_int32), ("dt", C.c_float), ("eps", C.c_float),
                ("omega_o", C.c_float * 3), ("seed", C.c_uint64), ("ff_signed", C.c_int32),
                ("extrap_order", C.c_int32), ("r_min", C.c_float), ("r_max", C.c_float), ("rec_base", C.c_int64),
                ("parts", C.c_int32), ("lo_grad", C.c_int32)]


class RecordsView(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("L", "grad", "hess", "L_ss", "grad_ss", "hess_ss", "L_ms", "grad_ms",
                                           "hess_ms", "L_ff", "radius", "eig", "kappa", "status", "pos",
                                           "n_cells", "n_far", "n_shells", "log_radius", "hit_prim", "hit_t")] + [("dbg_stride", C.c_int32)] + \
        [("radii", C.c_void_p), ("axes", C.c_void_p), ("dbg_lit", C.c_void_p), ("dbg_shells", C.c_int32)]


class RecordTuning(C.Structure):
    _fields_ = [("threads", C.c_int32), ("chunk_bands", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("shadow_bvh", C.c_int32), ("no_prepass", C.c_int32)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libvrc.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise VrcError(f"libvrc.so not built ({p}); run paper_1805_09258_gb300.build.build()")
    L = C.CDLL(p)
    P, I32 = C.c_void_p, C.c_int32
    L.vrc_build_scene.argtypes = [P, I32, P, I32, P, P, P, P, I32, C.POINTER(C.c_void_p)]
    L.vrc_destroy_scene.argtypes = [P]
    L.vrc_destroy_scene.restype = None
    L.vrc_compute_records.argtypes = [P, P, I32, P, P, P, P]
    L.vrc_compute_records_host.argtypes = [P, P, I32, P, P, P, P, P, P]
    L.vrc_cache_step_host.argtypes = [P, C.POINTER(C.c_void_p), P, I32, P, P, I32, P, P, P, P, P, P, P]
    L.vrc_set_record_tuning.argtypes = [P, P]
    L.vrc_record_timing.argtypes = [P, I32]
    L.vrc_record_kernel_times.argtypes = [P, P, P]
    L.vrc_autotune_records.argtypes = [P, P, I32, P, P, P, P, P]
    L.vrc_records_graph_create.argtypes = [P, P, I32, P, P, P, C.POINTER(C.c_void_p)]
    L.vrc_graph_launch.argtypes = [P, P]
    L.vrc_graph_destroy.argtypes = [P]
    L.vrc_graph_destroy.restype = None
    L.vrc_get_record_tuning.argtypes = [P, P]
    L.vrc_build_record_grid.argtypes = [P, I32, I32, C.POINTER(C.c_void_p), P]
    L.vrc2d_build_scene.argtypes = [P, I32, P, C.c_float, C.c_float, P, I32, C.POINTER(C.c_void_p)]
    L.vrc2d_destroy_scene.argtypes = [P]
    L.vrc2d_destroy_scene.restype = None
    L.vrc2d_compute_records.argtypes = [P, P, I32, P, P, P]
    L.vrc_build_record_grid_aniso.argtypes = [P, I32, I32, C.POINTER(C.c_void_p), P]
    L.vrc_rebuild_record_grid.argtypes = [P, P, I32, I32, I32, P]
    L.vrc_destroy_grid.argtypes = [P]
    L.vrc_destroy_grid.restype = None
    L.vrc_query_inscatter.argtypes = [P, P, I32, P, P, P]
    L.vrc_query_inscatter_noalloc.argtypes = [P, I32, I32, P, I32, P, P, P]
    L.vrc_coarse_features.argtypes = [P, P, I32, P, P, P]
    L.vrc_coarse_features_bf16.argtypes = [P, P, I32, P, P, P]
    L.vrc_march_points.argtypes = [P, P, I32, I32, I32, I32, I32, I32, P, P, P]
    L.vrc_render.argtypes = [P, P, P, P, I32, I32, I32, I32, I32, P, P, P]
    L.vrc_composite.argtypes = [P, P, I32, I32, I32, I32, I32, P, P, P]
    L.vrc_select_sites.argtypes = [P, P, I32, I32, P, C.c_int64, P, P, P, P, P]
    L.vrc_select_sites_levels.argtypes = [P, P, I32, I32, I32, P, C.c_int64, P, P, P, P, P]
    L.vrc_bump_levels.argtypes = [P, I32, I32, P]
    L.vrc_update_coverage.argtypes = [P, I32, P, P]
    L.vrc_init_levels.argtypes = [P, I32, I32, P, P]
    L.vrc_march_pixels.argtypes = [P, P, P, I32, I32, P, P, P]
    L.vrc_render_pixels.argtypes = [P, P, P, P, P, I32, I32, P, P, P]
    L.vrc_compact_indices.argtypes = [P, I32, P, C.c_int64, P, P, P]
    L.vrc_levels_by_cell.argtypes = [P, I32, I32, P, P, P, I32, C.c_float, I32, I32, P, P, P]
    L.vrc_levels_from_radius.argtypes = [P, I32, C.c_float, I32, I32, P, P]
    L.vrc_retire_level.argtypes = [P, I32, I32, P]
    L.vrc_mlp_fallback.argtypes = [P, I32, C.c_float, P, C.c_float, P, P, P]
    L.vrc_mlp_create.argtypes = [P, C.POINTER(C.c_void_p)]
    L.vrc_mlp_destroy.argtypes = [P]
    L.vrc_mlp_destroy.restype = None
    L.vrc_mlp_num_params.restype = I32
    L.vrc_mlp_get_params.argtypes = [P, P, P, P, P]
    L.vrc_mlp_set_params.argtypes = [P, P, P, P, C.c_int64]
    L.vrc_mlp_predict.argtypes = [P, P, I32, P, P]
    L.vrc_mlp_predict_bf16.argtypes = [P, P, I32, P, P]
    L.vrc_mlp_gradient.argtypes = [P, P, P, I32, P, P, P]
    L.vrc_mlp_train_step.argtypes = [P, P, P, I32, C.c_float, C.c_float, P, P]
    L.vrc_mlp_status.argtypes = [P]
    L.vrc_status_string.restype = C.c_char_p
    L.vrc_status_string.argtypes = [C.c_int]
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != VRC_OK:
        msg = load_library().vrc_status_string(rc).decode()
        raise VrcError(f"{what} failed: {msg} ({rc})")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise VrcError("no CUDA device: libvrc runs on the GPU only")
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def record_params(rp) -> RecordParamsC:
    """Marshal any object with the RecordParams fields into the C struct."""
    p = RecordParamsC()
    p.n_bands, p.n_bins = int(rp.n_bands), int(rp.n_bins)
    p.dt, p.eps = float(rp.dt), float(rp.eps)
    p.omega_o[:] = [float(v) for v in rp.omega_o]
    p.seed = int(rp.seed)
    p.ff_signed, p.extrap_order = int(rp.ff_signed), int(rp.extrap_order)
    p.r_min, p.r_max = float(rp.r_min), float(rp.r_max)
    p.rec_base = int(getattr(rp, "rec_base", 0))
    p.parts = int(getattr(rp, "parts", 0))
    p.lo_grad = int(getattr(rp, "lo_grad", 0))
    return p


class Scene:
    """A scene on the device (vrc_build_scene / vrc_destroy_scene)."""

    def __init__(self, tris, albedo, medium, lights, emission=None):
        L = load_library()
        tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 3, 3)
        n = tris.shape[0]
        verts = np.ascontiguousarray(tris.reshape(-1, 3))
        idx = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
        albedo = np.ascontiguousarray(albedo, dtype=np.float32).reshape(n, 3)
        em = None if emission is None else np.ascontiguousarray(emission, dtype=np.float32).reshape(n, 3)
        med = _Medium(float(medium.sigma_s), float(medium.sigma_a), float(medium.g))
        nl = len(lights)
        larr = (_Light * max(nl, 1))()
        for i, l in enumerate(lights):
            larr[i].pos[:] = [float(v) for v in l.pos]
            larr[i].intensity[:] = [float(v) for v in l.intensity]
        h = C.c_void_p()
        rc = L.vrc_build_scene(verts.ctypes.data, verts.shape[0], idx.ctypes.data, n, albedo.ctypes.data,
                               None if em is None else em.ctypes.data, C.byref(med), C.byref(larr), nl, C.byref(h))
        _check(rc, "vrc_build_scene")
        self.handle = h
        self.n_tris = n

    @classmethod
    def from_workload(cls, scene):
        return cls(scene.tris, scene.albedo, scene.medium, scene.lights, scene.emission)

    def record_timing(self, enable: bool = True):
        """vrc_record_timing: CUDA events around the kernels of each compute_records call."""
        _check(load_library().vrc_record_timing(self.handle, int(enable)), "vrc_record_timing")

    def kernel_times(self):
        """vrc_record_kernel_times: (summed ms of pre-pass, record kernel, radius stage; calls)."""
        ms = (C.c_float * 3)()
        n = C.c_int32(0)
        _check(load_library().vrc_record_kernel_times(self.handle, ms, C.byref(n)), "vrc_record_kernel_times")
        return [float(v) for v in ms], int(n.value)

    def set_tuning(self, threads=0, chunk_bands=0, blocks_per_sm=0, shadow_bvh=0, no_prepass=0):
        t = RecordTuning(threads, chunk_bands, blocks_per_sm, shadow_bvh, no_prepass)
        _check(load_library().vrc_set_record_tuning(self.handle, C.byref(t)), "vrc_set_record_tuning")

    def get_tuning(self):
        t = RecordTuning()
        _check(load_library().vrc_get_record_tuning(self.handle, C.byref(t)), "vrc_get_record_tuning")
        return dict(threads=t.threads, chunk_bands=t.chunk_bands, blocks_per_sm=t.blocks_per_sm,
                    shadow_bvh=t.shadow_bvh, no_prepass=t.no_prepass)

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.vrc_destroy_scene(self.handle)
                self.handle = None
        except Exception:
            pass


build_scene = Scene

RECORD_FIELDS = dict(L=3, grad=9, hess=18, L_ss=3, grad_ss=9, hess_ss=18, L_ms=3, grad_ms=9, hess_ms=18,
                     L_ff=3, radius=1, eig=3, kappa=1, pos=3)


def alloc_records(n: int, full: bool = True, device="cuda", aniso: bool = False):
    """Allocate the per-record output tensors (float32; status int32).  aniso (or full)
    adds the ellipsoid outputs radii [n,3] and axes [n,9]."""
    torch = _torch()
    out = {}
    for k, w in RECORD_FIELDS.items():
        if not full and k not in ("L", "grad", "hess", "radius", "pos"):
            continue
        out[k] = torch.empty((n, w) if w > 1 else (n,), dtype=torch.float32, device=device)
    if full or aniso:
        out["radii"] = torch.empty((n, 3), dtype=torch.float32, device=device)
        out["axes"] = torch.empty((n, 9), dtype=torch.float32, device=device)
    out["status"] = torch.empty((n,), dtype=torch.int32, device=device)
    if full:
        out["n_cells"] = torch.empty((n,), dtype=torch.int32, device=device)
        out["n_far"] = torch.empty((n,), dtype=torch.int32, device=device)
        out["n_shells"] = torch.empty((n,), dtype=torch.int32, device=device)
    return out


def records_view(out: dict, dbg_stride: int = 0) -> RecordsView:
    v = RecordsView()
    for k in ("L", "grad", "hess", "L_ss", "grad_ss", "hess_ss", "L_ms", "grad_ms", "hess_ms", "L_ff", "radius",
              "eig", "kappa", "status", "pos", "n_cells", "n_far", "n_shells", "log_radius", "hit_prim", "hit_t",
              "radii", "axes", "dbg_lit"):
        setattr(v, k, _ptr(out.get(k)))
    v.dbg_stride = dbg_stride
    if out.get("dbg_lit") is not None:
        v.dbg_shells = int(out["dbg_lit"].shape[1])
    return v


def compute_records(scene: Scene, pos, params, n_bands=None, out: Optional[dict] = None, full: bool = True,
                    debug_hits: bool = False, stream=None) -> dict:
    """vrc_compute_records on device positions `pos` [n,3] (float32 CUDA tensor)."""
    torch = _torch()
    assert pos.is_cuda and pos.dtype == torch.float32 and pos.is_contiguous()
    n = pos.shape[0]
    if out is None:
        out = alloc_records(n, full=full, device=pos.device)
    stride = 0
    if debug_hits:
        nb = int(params.n_bands)
        ns = 2 * nb if n_bands is not None else int(params.n_bins)
        stride = nb * ns + 2
        out["hit_prim"] = torch.full((n, stride), -2, dtype=torch.int32, device=pos.device)
        out["hit_t"] = torch.zeros((n, stride), dtype=torch.float32, device=pos.device)
        # visibility decisions: a bit per (shell, ray); every ray ends inside the unit cube,
        # so shells beyond ceil(sqrt(3) / dt) hold no open vertex
        shells = int(math.ceil(math.sqrt(3.0) / float(params.dt))) + 2
        out["dbg_lit"] = torch.zeros((n, shells, (stride + 31) // 32), dtype=torch.int32, device=pos.device)
    v = records_view(out, stride)
    p = record_params(params)
    nbp = None
    if n_bands is not None:
        assert n_bands.is_cuda and n_bands.dtype == torch.int32
        nbp = _ptr(n_bands)
    rc = load_library().vrc_compute_records(scene.handle, _ptr(pos), n, nbp, C.byref(p), C.byref(v),
                                            _stream_ptr(stream))
    _check(rc, "vrc_compute_records")
    return out


class _Light2(C.Structure):
    _fields_ = [("pos", C.c_float * 2), ("intensity", C.c_float * 3)]


class Scene2D:
    """A scene of the 2D world on the device (vrc2d_build_scene / vrc2d_destroy_scene):
    segments [n, 4] (x0, y0, x1, y1), albedo [n, 3], medium sigma_s / sigma_a, point lights
    with .pos (2) and .intensity (3)."""

    def __init__(self, segs, albedo, sigma_s, sigma_a, lights):
        L = load_library()
        segs = np.ascontiguousarray(segs, dtype=np.float32).reshape(-1, 4)
        n = segs.shape[0]
        albedo = np.ascontiguousarray(albedo, dtype=np.float32).reshape(n, 3)
        nl = len(lights)
        larr = (_Light2 * max(nl, 1))()
        for i, l in enumerate(lights):
            larr[i].pos[:] = [float(v) for v in l.pos]
            larr[i].intensity[:] = [float(v) for v in l.intensity]
        h = C.c_void_p()
        rc = L.vrc2d_build_scene(segs.ctypes.data if n else None, n, albedo.ctypes.data if n else None,
                                 float(sigma_s), float(sigma_a), C.byref(larr), nl, C.byref(h))
        _check(rc, "vrc2d_build_scene")
        self.handle = h
        self.n_segs = n

    @classmethod
    def from_workload(cls, scene):
        return cls(scene.segs, scene.albedo, scene.sigma_s, scene.sigma_a, scene.lights)

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.vrc2d_destroy_scene(self.handle)
                self.handle = None
        except Exception:
            pass


def compute_records_2d(scene: Scene2D, pos, params, out: Optional[dict] = None, full: bool = True,
                       debug_hits: bool = False, stream=None) -> dict:
    """vrc2d_compute_records on device positions pos [n, 2]: records in the 3D layout in
    the plane z = 0.5 (see vrc.h).  debug_hits: also each ray's hit segment and t."""
    torch = _torch()
    assert pos.is_cuda and pos.dtype == torch.float32 and pos.is_contiguous() and pos.shape[1] == 2
    n = pos.shape[0]
    if out is None:
        out = alloc_records(n, full=full, device=pos.device)
    stride = 0
    if debug_hits:
        stride = int(params.n_bins)
        out["hit_prim"] = torch.full((n, stride), -2, dtype=torch.int32, device=pos.device)
        out["hit_t"] = torch.zeros((n, stride), dtype=torch.float32, device=pos.device)
    v = records_view(out, stride)
    p = record_params(params)
    rc = load_library().vrc2d_compute_records(scene.handle, _ptr(pos), n, C.byref(p), C.byref(v),
                                              _stream_ptr(stream))
    _check(rc, "vrc2d_compute_records")
    return out


def autotune_records(scene: Scene, pos, params, out: dict, n_bands=None, stream=None) -> dict:
    """vrc_autotune_records: pick the record kernel's launch shape by timing; returns it."""
    t = RecordTuning()
    v = records_view(out)
    p = record_params(params)
    rc = load_library().vrc_autotune_records(scene.handle, _ptr(pos), pos.shape[0], _ptr(n_bands), C.byref(p),
                                             C.byref(v), _stream_ptr(stream), C.byref(t))
    _check(rc, "vrc_autotune_records")
    return dict(threads=t.threads, chunk_bands=t.chunk_bands, blocks_per_sm=t.blocks_per_sm, shadow_bvh=t.shadow_bvh,
                no_prepass=t.no_prepass)


class RecordsGraph:
    """A CUDA graph of one compute_records call on fixed buffers (vrc_records_graph_create)."""

    def __init__(self, scene: Scene, pos, params, out: dict, n_bands=None):
        self._keep = (scene, pos, out, n_bands)
        v = records_view(out)
        p = record_params(params)
        h = C.c_void_p()
        rc = load_library().vrc_records_graph_create(scene.handle, _ptr(pos), pos.shape[0], _ptr(n_bands),
                                                     C.byref(p), C.byref(v), C.byref(h))
        _check(rc, "vrc_records_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(load_library().vrc_graph_launch(self.handle, _stream_ptr(stream)), "vrc_graph_launch")

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.vrc_graph_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def compute_records_host(scene: Scene, pos: np.ndarray, params) -> dict:
    """vrc_compute_records_host: host positions in, host arrays out (synchronous)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
    n = pos.shape[0]
    res = dict(L=np.zeros((n, 3), np.float32), grad=np.zeros((n, 9), np.float32),
               hess=np.zeros((n, 18), np.float32), radius=np.zeros(n, np.float32), status=np.zeros(n, np.int32))
    p = record_params(params)
    rc = load_library().vrc_compute_records_host(scene.handle, pos.ctypes.data, n, C.byref(p),
                                                 res["L"].ctypes.data, res["grad"].ctypes.data,
                                                 res["hess"].ctypes.data, res["radius"].ctypes.data,
                                                 res["status"].ctypes.data)
    _check(rc, "vrc_compute_records_host")
    return res


def _host_ptr(a):
    """Address of a host buffer: a numpy array or a (page-locked) torch CPU tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda and a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class HostStep:
    """vrc_cache_step_host: one whole step from host buffers -- records at host positions,
    the record grid (built on the first call, rebuilt in place after), queries at host
    points -- with the copies inside the call.  Host buffers may be numpy arrays or
    page-locked torch CPU tensors (the copies overlap the kernels only when page-locked)."""

    def __init__(self, scene: "Scene", params):
        self.scene = scene
        self.params = params
        self._grid = C.c_void_p()

    def __call__(self, pos, q, out: dict) -> dict:
        """pos [n, 3], q [nq, 3] float32 host buffers; out: host buffers L [n, 3], grad [n, 9],
        hess [n, 18], radius [n], status [n] (any may be missing), rgb [nq, 3], qstatus [nq]."""
        n, nq = int(pos.shape[0]), int(q.shape[0])
        p = record_params(self.params)
        rc = load_library().vrc_cache_step_host(self.scene.handle, C.byref(self._grid), _host_ptr(pos), n,
                                                C.byref(p), _host_ptr(q), nq,
                                                *[_host_ptr(out.get(k)) for k in ("L", "grad", "hess", "radius",
                                                                                  "status", "rgb", "qstatus")])
        _check(rc, "vrc_cache_step_host")
        return out

    def __del__(self):
        try:
            if self._grid:
                load_library().vrc_destroy_grid(self._grid)
        except Exception:
            pass


class Grid:
    """Record lookup structure (vrc_build_record_grid / vrc_build_record_grid_aniso /
    vrc_destroy_grid).  aniso=True uses the records' ellipsoids (radii, axes)."""

    def __init__(self, records: dict, n: Optional[int] = None, extrap_order: int = 1, stream=None,
                 aniso: bool = False):
        n = records["L"].shape[0] if n is None else n
        v = records_view(records)
        h = C.c_void_p()
        self._keep = records
        fn = "vrc_build_record_grid_aniso" if aniso else "vrc_build_record_grid"
        rc = getattr(load_library(), fn)(C.byref(v), n, extrap_order, C.byref(h), _stream_ptr(stream))
        _check(rc, fn)
        self.handle = h
        self.n = n
        self.extrap_order = extrap_order
        self.aniso = aniso

    def rebuild(self, records: dict, n: Optional[int] = None, stream=None):
        """vrc_rebuild_record_grid: the same grid object rebuilt from new records, reusing
        its device buffers."""
        n = records["L"].shape[0] if n is None else n
        v = records_view(records)
        self._keep = records
        rc = load_library().vrc_rebuild_record_grid(self.handle, C.byref(v), n, self.extrap_order, int(self.aniso),
                                                    _stream_ptr(stream))
        _check(rc, "vrc_rebuild_record_grid")
        self.n = n
        return self

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.vrc_destroy_grid(self.handle)
                self.handle = None
        except Exception:
            pass


build_record_grid = Grid


def query_inscatter(grid: Grid, q, rgb=None, status=None, stream=None):
    """vrc_query_inscatter on device query points q [nq,3]; returns (rgb [nq,3], count [nq])."""
    torch = _torch()
    assert q.is_cuda and q.dtype == torch.float32 and q.is_contiguous()
    nq = q.shape[0]
    if rgb is None:
        rgb = torch.empty((nq, 3), dtype=torch.float32, device=q.device)
    if status is None:
        status = torch.empty((nq,), dtype=torch.int32, device=q.device)
    rc = load_library().vrc_query_inscatter(grid.handle, _ptr(q), nq, _ptr(rgb), _ptr(status), _stream_ptr(stream))
    _check(rc, "vrc_query_inscatter")
    return rgb, status


NOALLOC_MAX_RECORDS = 65536


def query_inscatter_noalloc(records: dict, q, n: Optional[int] = None, extrap_order: int = 1, rgb=None,
                            status=None, stream=None):
    """vrc_query_inscatter_noalloc: the same queries without a grid object.

    For callers that cannot allocate device memory at query time: the library uses a
    fixed 4 MiB device array instead of cudaMalloc.  Calls that overlap on the GPU race
    on that array; keep them ordered on one stream.  The first call on a device may load
    the library's device code and reserve the array (CUDA loads modules lazily): make it
    during start-up, before any stream capture.  Sphere records only (radii and axes are
    ignored).
    """
    torch = _torch()
    assert q.is_cuda and q.dtype == torch.float32 and q.is_contiguous()
    n = records["L"].shape[0] if n is None else n
    nq = q.shape[0]
    if rgb is None:
        rgb = torch.empty((nq, 3), dtype=torch.float32, device=q.device)
    if status is None:
        status = torch.empty((nq,), dtype=torch.int32, device=q.device)
    v = records_view(records)
    rc = load_library().vrc_query_inscatter_noalloc(C.byref(v), n, extrap_order, _ptr(q), nq, _ptr(rgb),
                                                    _ptr(status), _stream_ptr(stream))
    _check(rc, "vrc_query_inscatter_noalloc")
    return rgb, status


def coarse_features(scene: Scene, pos, params, out=None, stream=None, bf16: bool = False):
    """vrc_coarse_features (vrc_coarse_features_bf16 with bf16=True): [n, 2 N] features of
    the coarse ray set at `pos`, float32 (or bfloat16)."""
    torch = _torch()
    n = pos.shape[0]
    N = int(params.n_bands) * int(params.n_bins)
    if out is None:
        out = torch.empty((n, 2 * N), dtype=torch.bfloat16 if bf16 else torch.float32, device=pos.device)
    p = record_params(params)
    fn = "vrc_coarse_features_bf16" if out.dtype == torch.bfloat16 else "vrc_coarse_features"
    _check(getattr(load_library(), fn)(scene.handle, _ptr(pos), n, C.byref(p), _ptr(out), _stream_ptr(stream)), fn)
    return out


class MLP:
    """The learned radius predictor (vrc_mlp_*): 256-64-64-1 GELU network on tensor cores."""

    def __init__(self, params: np.ndarray):
        L = load_library()
        self.n_params = int(L.vrc_mlp_num_params())
        params = np.ascontiguousarray(params, dtype=np.float32)
        assert params.size == self.n_params
        h = C.c_void_p()
        _check(L.vrc_mlp_create(params.ctypes.data, C.byref(h)), "vrc_mlp_create")
        self.handle = h

    def get_params(self, with_moments: bool = False):
        p = np.zeros(self.n_params, np.float32)
        m = np.zeros(self.n_params, np.float32) if with_moments else None
        v = np.zeros(self.n_params, np.float32) if with_moments else None
        step = C.c_int64(0)
        _check(load_library().vrc_mlp_get_params(self.handle, p.ctypes.data, None if m is None else m.ctypes.data,
                                                 None if v is None else v.ctypes.data, C.byref(step)),
               "vrc_mlp_get_params")
        return (p, m, v, step.value) if with_moments else p

    def set_params(self, p, m=None, v=None, step: int = 0):
        p = np.ascontiguousarray(p, dtype=np.float32)
        m = None if m is None else np.ascontiguousarray(m, dtype=np.float32)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        _check(load_library().vrc_mlp_set_params(self.handle, p.ctypes.data, None if m is None else m.ctypes.data,
                                                 None if v is None else v.ctypes.data, step), "vrc_mlp_set_params")

    def predict(self, feat, out=None, stream=None):
        """Predicted log radius per feature row: float32 features through vrc_mlp_predict,
        bfloat16 features through vrc_mlp_predict_bf16 (tiled TMA copies)."""
        torch = _torch()
        n = feat.shape[0]
        assert feat.is_cuda and feat.is_contiguous()
        if out is None:
            out = torch.empty((n,), dtype=torch.float32, device=feat.device)
        fn = "vrc_mlp_predict_bf16" if feat.dtype == torch.bfloat16 else "vrc_mlp_predict"
        _check(getattr(load_library(), fn)(self.handle, _ptr(feat), n, _ptr(out), _stream_ptr(stream)), fn)
        return out

    def gradient(self, feat, target, stream=None):
        torch = _torch()
        g = torch.empty((self.n_params,), dtype=torch.float32, device=feat.device)
        pred = torch.empty((feat.shape[0],), dtype=torch.float32, device=feat.device)
        _check(load_library().vrc_mlp_gradient(self.handle, _ptr(feat), _ptr(target), feat.shape[0], _ptr(g),
                                               _ptr(pred), _stream_ptr(stream)), "vrc_mlp_gradient")
        return g, pred

    def train_step(self, feat, target, lr: float, weight_decay: float = 1e-4, want_loss: bool = False,
                   stream=None):
        loss = C.c_float(0.0)
        _check(load_library().vrc_mlp_train_step(self.handle, _ptr(feat), _ptr(target), feat.shape[0], lr,
                                                 weight_decay, C.byref(loss) if want_loss else None,
                                                 _stream_ptr(stream)), "vrc_mlp_train_step")
        return loss.value if want_loss else None

    def status(self) -> int:
        return int(load_library().vrc_mlp_status(self.handle))

    def __del__(self):
        try:
            if getattr(self, "handle", None) and _lib is not None:
                _lib.vrc_mlp_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("forward", C.c_float * 3), ("vfov_deg", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32)]

    @classmethod
    def make(cls, pos, forward, vfov_deg, width, height):
        c = cls()
        c.pos[:] = [float(v) for v in pos]
        c.forward[:] = [float(v) for v in forward]
        c.vfov_deg, c.width, c.height = float(vfov_deg), int(width), int(height)
        return c


def march_points(scene: Scene, cam: Camera, x0, y0, w, h, stride, steps, stream=None):
    torch = _torch()
    n = w * h * steps
    pts = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    valid = torch.empty((n,), dtype=torch.int32, device="cuda")
    _check(load_library().vrc_march_points(scene.handle, C.byref(cam), x0, y0, w, h, stride, steps, _ptr(pts),
                                           _ptr(valid), _stream_ptr(stream)), "vrc_march_points")
    return pts, valid


def render(scene: Scene, grid: "Grid", cam: Camera, x0, y0, w, h, steps, img=None, miss=None, stream=None,
           grid2: "Grid" = None):
    """vrc_render; grid2 (optional) is a second cache whose look-up is added (separate
    single- and multiple-scattering caches)."""
    torch = _torch()
    if img is None:
        img = torch.empty((w * h, 3), dtype=torch.float32, device="cuda")
    if miss is None:
        miss = torch.empty((w * h,), dtype=torch.int32, device="cuda")
    g2 = grid2.handle if grid2 is not None else None
    _check(load_library().vrc_render(scene.handle, grid.handle, g2, C.byref(cam), x0, y0, w, h, steps, _ptr(img),
                                     _ptr(miss), _stream_ptr(stream)), "vrc_render")
    return img, miss


def march_pixels(scene: Scene, cam: Camera, pix, steps, stream=None):
    torch = _torch()
    n = pix.shape[0] * steps
    pts = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    valid = torch.empty((n,), dtype=torch.int32, device="cuda")
    _check(load_library().vrc_march_pixels(scene.handle, C.byref(cam), _ptr(pix), pix.shape[0], steps, _ptr(pts),
                                           _ptr(valid), _stream_ptr(stream)), "vrc_march_pixels")
    return pts, valid


def render_pixels(scene: Scene, grid: "Grid", cam: Camera, pix, steps, img, miss, stream=None, grid2: "Grid" = None):
    g2 = grid2.handle if grid2 is not None else None
    _check(load_library().vrc_render_pixels(scene.handle, grid.handle, g2, C.byref(cam), _ptr(pix), pix.shape[0],
                                            steps, _ptr(img), _ptr(miss), _stream_ptr(stream)), "vrc_render_pixels")


def compact_indices(flags, scratch, out, stream=None) -> int:
    cnt = C.c_int32(0)
    _check(load_library().vrc_compact_indices(_ptr(flags), flags.shape[0], _ptr(scratch), scratch.numel(), _ptr(out),
                                              C.byref(cnt), _stream_ptr(stream)), "vrc_compact_indices")
    return int(cnt.value)


def composite(scene: Scene, cam: Camera, x0, y0, w, h, steps, L, stream=None):
    torch = _torch()
    img = torch.empty((w * h, 3), dtype=torch.float32, device="cuda")
    _check(load_library().vrc_composite(scene.handle, C.byref(cam), x0, y0, w, h, steps, _ptr(L), _ptr(img),
                                        _stream_ptr(stream)), "vrc_composite")
    return img


def select_sites(pts, level, wave_level: int, scratch, site_idx, site_pts, stream=None, with_pool: bool = False):
    """vrc_select_sites: the number of sites; with_pool: (sites, candidates left in the pool)."""
    cnt, pool = C.c_int32(0), C.c_int32(0)
    _check(load_library().vrc_select_sites(_ptr(pts), _ptr(level), pts.shape[0], wave_level, _ptr(scratch),
                                           scratch.numel(), _ptr(site_idx), _ptr(site_pts), C.byref(cnt),
                                           C.byref(pool) if with_pool else None, _stream_ptr(stream)),
           "vrc_select_sites")
    return (int(cnt.value), int(pool.value)) if with_pool else int(cnt.value)


def select_sites_levels(pts, level, lmin: int, lmax: int, scratch, site_idx, site_pts, stream=None):
    """vrc_select_sites_levels: (sites, candidates left in the pool)."""
    cnt, pool = C.c_int32(0), C.c_int32(0)
    _check(load_library().vrc_select_sites_levels(_ptr(pts), _ptr(level), pts.shape[0], lmin, lmax, _ptr(scratch),
                                                  scratch.numel(), _ptr(site_idx), _ptr(site_pts), C.byref(cnt),
                                                  C.byref(pool), _stream_ptr(stream)), "vrc_select_sites_levels")
    return int(cnt.value), int(pool.value)


def bump_levels(level, lmax: int, stream=None):
    _check(load_library().vrc_bump_levels(_ptr(level), level.shape[0], lmax, _stream_ptr(stream)), "vrc_bump_levels")


def levels_by_cell(pts, cell_level: int, scratch, site_idx, site_logr, n_sites: int, cell_over_radius: float,
                   lmin: int, lmax: int, rep_level, level, stream=None):
    _check(load_library().vrc_levels_by_cell(_ptr(pts), pts.shape[0], cell_level, _ptr(scratch), _ptr(site_idx),
                                             _ptr(site_logr), n_sites, cell_over_radius, lmin, lmax, _ptr(rep_level),
                                             _ptr(level), _stream_ptr(stream)), "vrc_levels_by_cell")


def init_levels(valid, level, start_level: int, stream=None):
    _check(load_library().vrc_init_levels(_ptr(valid), valid.shape[0], start_level, _ptr(level), _stream_ptr(stream)),
           "vrc_init_levels")


def update_coverage(count, level, stream=None):
    _check(load_library().vrc_update_coverage(_ptr(count), count.shape[0], _ptr(level), _stream_ptr(stream)),
           "vrc_update_coverage")


def retire_level(level, lv: int, stream=None):
    _check(load_library().vrc_retire_level(_ptr(level), level.shape[0], lv, _stream_ptr(stream)), "vrc_retire_level")


def mlp_fallback(logr, logr_offset: float, radius_coarse, logr_fallback: float, out=None, n_fallback=None,
                 stream=None):
    """vrc_mlp_fallback: the predicted log radius shifted by logr_offset, kept only where
    the coarse record's radius is at least that (radius_coarse None: shift only); returns
    (logr_out, n_fallback device int32[1])."""
    torch = _torch()
    n = logr.shape[0]
    out = torch.empty_like(logr) if out is None else out
    if n_fallback is None:
        n_fallback = torch.zeros((1,), dtype=torch.int32, device=logr.device)
    _check(load_library().vrc_mlp_fallback(_ptr(logr), n, float(logr_offset), _ptr(radius_coarse),
                                           float(logr_fallback), _ptr(out), _ptr(n_fallback), _stream_ptr(stream)),
           "vrc_mlp_fallback")
    return out, n_fallback


def levels_from_radius(logr, level, cell_over_radius: float, lmin: int, lmax: int, stream=None):
    _check(load_library().vrc_levels_from_radius(_ptr(logr), logr.shape[0], cell_over_radius, lmin, lmax,
                                                 _ptr(level), _stream_ptr(stream)), "vrc_levels_from_radius")
