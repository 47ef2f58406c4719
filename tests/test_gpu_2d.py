"""GPU parity of the 2D world's records (Sec. 3; Sec. 4 in 2D; App. A, App. B, Eq.
radiusAniso2D) against the FP64 2D oracle, through the C ABI: the small scene in full,
the mid scene at full size (4,096 records x 512 directions) with a seeded sample, the
single- / multiple-scattering parts, and 2D queries through the 3D record grid in the
plane z = 0.5.

Tolerances as for 3D records: radiance 1e-4 relative, gradient and Hessian 1e-3 of
their norms, plus each record's decision budget (the change that flipping its near-tie
shadow or clamp decisions could make, computed by the oracle).  The oracle takes the
GPU's primary hit segments (replay mode), so records whose primary rays pass within 1e-5
of a segment endpoint, where FP32 and FP64 may see different segments, are compared too."""
import numpy as np
import pytest

import oracle as O
import oracle.world2d as O2
from tests.gpu_helpers import TOL_D, TOL_L, to_np
from workloads import flat

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

Y = np.array([0.2126, 0.7152, 0.0722])


@pytest.fixture(scope="module")
def vrc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_09258_gb300 import build
    build.build()
    import paper_1805_09258_gb300 as m
    return m


def gpu_records(vrc, w, pos, params=None, debug_hits=True):
    s = vrc.Scene2D.from_workload(w.scene)
    out = vrc.compute_records_2d(s, torch.from_numpy(np.ascontiguousarray(pos)).cuda(), params or w.params,
                                 debug_hits=debug_hits)
    torch.cuda.synchronize()
    return to_np(out)


def oracle2d(w, params, pos, g, idx=None):
    """The 2D oracle on the GPU's primary hit segments (replay mode)."""
    hits = g["hit_prim"] if idx is None else g["hit_prim"][idx]
    return O2.records(O2.OracleScene2(w.scene), params, pos if idx is None else pos[idx],
                      rec_ids=idx, replay_hits=hits)


def compare2d(g, ref, idx, sfx=""):
    fails, checked = [], 0
    for r, i in enumerate(idx):
        assert ref["prim_near"][r] == 0          # replay: no primary decision is open
        checked += 1
        Lg, Lo = g["L" + sfx][i].astype(np.float64), ref["L" + sfx][r]
        if np.any(np.abs(Lg - Lo) > TOL_L * np.abs(Lo) + ref["bud_L"][r] + 1e-12):
            fails.append((int(i), "L", Lg, Lo))
        gg = g["grad" + sfx][i].reshape(3, 3).astype(np.float64)
        hg = g["hess" + sfx][i].reshape(3, 6).astype(np.float64)
        assert np.all(gg[:, 2] == 0) and np.all(hg[:, [2, 4, 5]] == 0)
        for c in range(3):
            eg = np.linalg.norm(gg[c, :2] - ref["grad" + sfx][r, c])
            if eg > TOL_D * np.linalg.norm(ref["grad" + sfx][r, c]) + ref["bud_grad"][r, c] + 1e-12:
                fails.append((int(i), f"grad[{c}]", eg))
            ho = ref["hess" + sfx][r, c]
            dh = hg[c, [0, 1, 3]] - ho
            fro = lambda h: np.sqrt(h[0] ** 2 + 2 * h[1] ** 2 + h[2] ** 2)
            if fro(dh) > TOL_D * fro(ho) + ref["bud_hess"][r, c] + 1e-12:
                fails.append((int(i), f"hess[{c}]", fro(dh), fro(ho)))
    assert not fails, f"{len(fails)} mismatches, first: {fails[:5]}"
    return checked


def check_radius(g, ref, idx, p):
    for r, i in enumerate(idx):
        LY = float(Y @ ref["L"][r])
        hy = (Y[:, None] * ref["hess"][r]).sum(0)
        lam = np.abs(ref["eig"][r]).max()
        dH = TOL_D * np.sqrt(hy[0] ** 2 + 2 * hy[1] ** 2 + hy[2] ** 2) + float(Y @ ref["bud_hess"][r])
        dL = TOL_L * abs(LY) + float(Y @ ref["bud_L"][r])
        rel = 0.25 * (dL / max(abs(LY), 1e-30) + dH / max(lam, 1e-30)) + 1e-5
        Ro, Rg = ref["radius"][r], float(g["radius"][i])
        assert abs(Rg - Ro) <= rel * Ro * 1.5 + 1e-7, (int(i), Rg, Ro, rel)
        # the ellipse: its smaller in-plane radius is the record's radius, the normal axis r_max
        rr = np.sort(g["radii"][i])
        assert abs(rr[0] - Rg) <= 1e-6 * Rg
        ax = g["axes"][i].reshape(3, 3)
        zrow = int(np.argmax(np.abs(ax[:, 2])))
        rz = p.r_max if LY > 0 else p.r_min          # a black record is r_min on every axis
        assert abs(g["radii"][i, zrow] - rz) <= 1e-7 and abs(ax[zrow, 2]) == 1.0


def test_small_scene_all_records(vrc):
    w = flat.flat_small()
    pos = w.positions()
    g = gpu_records(vrc, w, pos)
    ref = oracle2d(w, w.params, pos, g)
    n = compare2d(g, ref, np.arange(pos.shape[0]))
    assert n == pos.shape[0]
    plain = gpu_records(vrc, w, pos, debug_hits=False)
    for k in ("L", "grad", "hess", "radius"):
        assert np.array_equal(plain[k], g[k]), k             # the debug output changes nothing
    for sfx in ("_ss", "_ms"):
        compare2d(g, ref, np.arange(pos.shape[0]), sfx)
    check_radius(g, ref, np.arange(pos.shape[0]), w.params)
    assert np.allclose(g["pos"][:, :2], pos) and np.all(g["pos"][:, 2] == np.float32(flat.Z_PLANE))
    assert np.array_equal(g["n_shells"], ref["n_shells"].astype(np.int32))


def test_mid_scene_full_size_sampled(vrc):
    w = flat.flat_mid()
    pos = w.positions()
    g = gpu_records(vrc, w, pos)
    idx = np.sort(np.random.default_rng(97).choice(pos.shape[0], 256, replace=False))
    ref = oracle2d(w, w.params, pos, g, idx)
    assert compare2d(g, ref, idx) == 256
    check_radius(g, ref, idx, w.params)
    assert np.isfinite(g["L"]).all() and (g["status"] & 1).sum() == 0


def test_ragged_direction_counts_and_parts(vrc):
    w = flat.flat_small()
    pos = w.positions(37, seed=13)
    for nd in (3, 129, 1000):
        p = W_replace(w.params, n_bins=nd)
        g = gpu_records(vrc, w, pos, p)
        ref = oracle2d(w, p, pos, g)
        compare2d(g, ref, np.arange(pos.shape[0]))
    whole = gpu_records(vrc, w, pos)
    for parts, sfx in ((1, "_ss"), (2, "_ms")):
        g = gpu_records(vrc, w, pos, W_replace(w.params, parts=parts), debug_hits=False)
        for k in ("L", "grad", "hess"):
            assert np.array_equal(g[k], whole[k + sfx]), (parts, k)


def W_replace(p, **kw):
    from dataclasses import replace
    return replace(p, **kw)


def test_invalid_arguments(vrc):
    w = flat.flat_small()
    pos = torch.from_numpy(w.positions(4)).cuda()
    s = vrc.Scene2D.from_workload(w.scene)
    for bad in (dict(n_bands=2), dict(n_bins=2), dict(parts=5), dict(dt=0.0)):
        with pytest.raises(vrc.VrcError):
            vrc.compute_records_2d(s, pos, W_replace(w.params, **bad))
    with pytest.raises(vrc.VrcError):
        vrc.Scene2D(np.array([[0.1, 0.1, 0.1, 0.1]], np.float32), np.ones((1, 3), np.float32), 0.8, 0.2, [])
    out = vrc.compute_records_2d(s, pos[:0].contiguous(), w.params)
    assert out["L"].shape[0] == 0


def test_2d_queries_through_the_record_grid(vrc):
    """2D records in the plane z = 0.5 answer 2D queries through the 3D grid and query
    kernel: the same as the oracle's Eq. radianceTaylor over the same records."""
    w = flat.flat_mid()
    pos = w.positions(1500, seed=21)
    g = gpu_records(vrc, w, pos)
    recs = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in ("pos", "L", "grad", "radius", "hess",
                                                                            "radii", "axes")}
    q2 = w.queries(50000, seed=22)
    q = np.concatenate([q2, np.full((q2.shape[0], 1), flat.Z_PLANE, np.float32)], axis=1)
    for aniso in (False, True):
        grid = vrc.Grid(recs, aniso=aniso)
        rgb, cnt = vrc.query_inscatter(grid, torch.from_numpy(q).cuda())
        rgb, cnt = rgb.cpu().numpy(), cnt.cpu().numpy()
        if aniso:
            from tests.test_gpu_aniso import oracle_metric
            ref, rc, near = O.query_aniso(g["pos"], oracle_metric({"radii": g["radii"], "axes": g["axes"]}), g["L"],
                                          g["grad"], None, q)
        else:
            ref, rc, near = O.query(g["pos"], g["radius"], g["L"], g["grad"], None, q)
        ok = near == 0
        assert np.array_equal(cnt[ok], rc[ok])
        hit = ok & (rc > 0)
        scale = np.abs(ref[hit]).max(axis=1, keepdims=True) + 1e-6
        assert np.all(np.abs(rgb[hit] - ref[hit]) <= 3e-5 * scale + 1e-7)
        assert hit.mean() > 0.5
