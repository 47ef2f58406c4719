"""GPU parity of ellipsoidal records (Eq. radiusAniso3D per eigenvalue; anisotropic cache
points, Sec. 6) against the FP64 oracle: the FP64 eigenvectors and principal radii the
record kernel writes, the ellipsoid grid, and the query and render look-ups over it.

Two levels of comparison for the records: (a) the eigen-solve and radii alone, with the
oracle fed the GPU's own radiance and Hessian (the same input to both: tight tolerance
on the region matrix M, which is unique even where eigenvectors are not); (b) end to
end against oracle records, where each principal radius must lie inside the interval
that the radiance and Hessian tolerances allow (Weyl: |d lambda_i| <= ||dH||_F)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import TOL_D, TOL_L, hess_fro, to_np

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


def gpu_records(vrc, w, pos):
    s = vrc.Scene.from_workload(w.scene)
    out = vrc.compute_records(s, torch.from_numpy(np.ascontiguousarray(pos)).cuda(), w.params)
    torch.cuda.synchronize()
    return to_np(out)


def region_matrix(radii, axes):
    axes = np.asarray(axes, np.float64).reshape(-1, 3, 3)
    r = np.asarray(radii, np.float64).reshape(-1, 3)
    return np.einsum("kij,ki,kil->kjl", axes, 1.0 / r ** 2, axes)


def check_stage(g, p):
    """(a) eigen-solve + radii from the GPU's own L and Hessian."""
    radii, axes, metric, lam, status = O.aniso_records(g["L"], g["hess"], p.eps, p.r_min, p.r_max)
    Mg = region_matrix(g["radii"], g["axes"])
    Mo = O.metric_matrix(metric)
    err = np.linalg.norm(Mg - Mo, axis=(1, 2)) / np.linalg.norm(Mo, axis=(1, 2))
    assert err.max() <= 2e-5, (int(err.argmax()), err.max())
    assert np.allclose(g["radii"], radii, rtol=2e-6)
    assert np.allclose(g["eig"], lam, rtol=1e-5, atol=1e-6 * np.abs(lam).max(axis=1, keepdims=True))
    # unit, orthogonal axes
    A = g["axes"].reshape(-1, 3, 3).astype(np.float64)
    assert np.allclose(A @ A.transpose(0, 2, 1), np.eye(3)[None], atol=1e-5)
    # the smallest principal radius is the isotropic radius
    assert np.allclose(g["radii"].min(axis=1), g["radius"], rtol=1e-6)


def radius_of(LY, lam, p):
    lam = np.abs(lam)
    with np.errstate(divide="ignore"):
        R = np.where(lam > 0, (15.0 * LY * p.eps / (4 * np.pi * np.maximum(lam, 1e-300))) ** 0.2, p.r_max)
    return np.clip(np.where(LY > 0, R, p.r_min), p.r_min, p.r_max)


def check_end_to_end(g, ref, idx, p):
    """(b) each principal radius within the interval the L and H tolerances allow."""
    o_radii, _, _, o_lam, _ = O.aniso_records(ref["L"], ref["hess"], p.eps, p.r_min, p.r_max)
    for r, i in enumerate(idx):
        LY = float(Y @ ref["L"][r])
        dLY = TOL_L * abs(LY) + float(Y @ ref["bud_L"][r])
        hy = (Y[:, None] * ref["hess"][r].reshape(3, 6)).sum(0)
        dH = TOL_D * hess_fro(hy) + float(Y @ ref["bud_hess"][r]) + 1e-12
        for a in range(3):
            lo_l, hi_l = max(abs(o_lam[r, a]) - dH, 0.0), abs(o_lam[r, a]) + dH
            R_hi = radius_of(LY + dLY, lo_l, p)
            R_lo = radius_of(max(LY - dLY, 0.0), hi_l, p)
            Rg = float(g["radii"][i, a])
            assert R_lo * (1 - 1e-5) <= Rg <= R_hi * (1 + 1e-5), (int(i), a, Rg, R_lo, R_hi, o_radii[r, a])


def test_small_workload_ellipsoids(vrc):
    w = W.config1()
    pos = w.positions()
    g = gpu_records(vrc, w, pos)
    check_stage(g, w.params)
    ref = O.records(O.OracleScene(w.scene), w.params, pos, track_margins=1)
    check_end_to_end(g, ref, np.arange(pos.shape[0]), w.params)
    # the ellipsoids are not spheres: their largest radius exceeds the smallest
    assert np.median(g["radii"].max(axis=1) / g["radii"].min(axis=1)) > 1.2


def test_mid_workload_ellipsoids_sampled(vrc):
    w = W.config2()
    pos = w.positions()
    g = gpu_records(vrc, w, pos)
    check_stage(g, w.params)                                     # every record of the launch
    idx = np.sort(np.random.default_rng(98).choice(pos.shape[0], 16, replace=False))
    ref = O.records(O.OracleScene(w.scene), w.params, pos[idx], rec_ids=idx, track_margins=1)
    check_end_to_end(g, ref, idx, w.params)


def synthetic_ellipsoids(n, seed):
    rng = np.random.default_rng(seed)
    axes = np.zeros((n, 3, 3))
    for k in range(n):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        axes[k] = (q * np.sign(np.diag(r))).T               # rows = unit axes
    tab = dict(pos=rng.uniform(0.0, 1.0, (n, 3)), radii=rng.uniform(0.02, 0.3, (n, 3)),
               axes=axes.reshape(n, 9), L=rng.uniform(0.05, 1.0, (n, 3)), grad=rng.normal(size=(n, 9)) * 0.5,
               hess=rng.normal(size=(n, 18)) * 2.0)
    return {k: np.ascontiguousarray(v.astype(np.float32)) for k, v in tab.items()}


def oracle_metric(tab):
    M = region_matrix(tab["radii"], tab["axes"])
    return np.stack([M[:, 0, 0], M[:, 0, 1], M[:, 0, 2], M[:, 1, 1], M[:, 1, 2], M[:, 2, 2]], axis=1)


def gpu_query(vrc, tab, q, order):
    recs = {k: torch.from_numpy(v).cuda() for k, v in tab.items()}
    grid = vrc.Grid(recs, extrap_order=order, aniso=True)
    rgb, cnt = vrc.query_inscatter(grid, torch.from_numpy(np.ascontiguousarray(q)).cuda())
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), cnt.cpu().numpy()


def check_query(rgb, cnt, ref, rc, near):
    ok = near == 0
    assert np.array_equal(cnt[ok], rc[ok])
    assert np.all(np.abs(cnt[~ok] - rc[~ok]) <= 2)
    hit = ok & (rc > 0)
    scale = np.abs(ref[hit]).max(axis=1, keepdims=True) + np.abs(ref[hit]) + 1e-6
    assert np.all(np.abs(rgb[hit] - ref[hit]) <= 3e-5 * scale + 1e-6)
    assert np.all(rgb[rc == 0] == 0)


@pytest.mark.parametrize("order", [1, 2])
def test_ellipsoid_query_parity(vrc, order):
    tab = synthetic_ellipsoids(700, seed=31)
    rng = np.random.default_rng(32)
    # uniform points, record centres, points just inside / outside principal axes, a corner
    ax = tab["axes"].reshape(-1, 3, 3)
    edge = np.concatenate([tab["pos"][:40] + (1 - 1e-3) * tab["radii"][:40, :1] * ax[:40, 0],
                           tab["pos"][:40] + (1 + 1e-3) * tab["radii"][:40, 2:3] * ax[:40, 2]])
    q = np.concatenate([rng.uniform(0, 1, (30000, 3)), tab["pos"][:50], edge,
                        rng.uniform(0.98, 1.0, (100, 3))]).astype(np.float32)
    rgb, cnt = gpu_query(vrc, tab, q, order)
    ref, rc, near = O.query_aniso(tab["pos"], oracle_metric(tab), tab["L"], tab["grad"], tab["hess"], q, order)
    check_query(rgb, cnt, ref, rc, near)
    assert cnt.max() > 1 and (cnt == 0).any()


def test_ellipsoid_grid_ragged_and_degenerate(vrc):
    for n, seed in ((1, 41), (33, 42), (5000, 43)):
        tab = synthetic_ellipsoids(n, seed)
        if n == 33:                                   # spheres and very flat ellipsoids
            tab["radii"][:10] = tab["radii"][:10, :1]
            tab["radii"][10:20, 0] = 1e-3
        q = np.random.default_rng(seed + 100).uniform(0, 1, (4099, 3)).astype(np.float32)
        rgb, cnt = gpu_query(vrc, tab, q, 1)
        ref, rc, near = O.query_aniso(tab["pos"], oracle_metric(tab), tab["L"], tab["grad"], None, q, 1)
        check_query(rgb, cnt, ref, rc, near)
    # empty table: every query misses
    empty = {k: v[:0] for k, v in synthetic_ellipsoids(1, 44).items()}
    rgb, cnt = gpu_query(vrc, empty, np.full((7, 3), 0.5, np.float32), 1)
    assert np.all(cnt == 0) and np.all(rgb == 0)


def test_grid_requires_ellipsoid_outputs(vrc):
    tab = synthetic_ellipsoids(8, 45)
    recs = {k: torch.from_numpy(v).cuda() for k, v in tab.items() if k != "axes"}
    with pytest.raises(vrc.VrcError):
        vrc.Grid(recs, aniso=True)


def test_ellipsoids_cover_more_than_spheres(vrc):
    """Records of the mid workload: every point inside a record's sphere (smallest radius)
    is inside its ellipsoid, so the ellipsoid grid answers at least as many queries."""
    w = W.config2()
    pos = w.positions(512, seed=7)
    g = gpu_records(vrc, w, pos)
    recs = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda() for k in ("pos", "L", "grad", "radius", "radii",
                                                                            "axes")}
    q = torch.from_numpy(w.queries(200000, seed=8)).cuda()
    _, c_iso = vrc.query_inscatter(vrc.Grid(recs), q)
    _, c_ell = vrc.query_inscatter(vrc.Grid(recs, aniso=True), q)
    c_iso, c_ell = c_iso.cpu().numpy(), c_ell.cpu().numpy()
    assert np.all(c_ell >= c_iso - 1)           # float rounding at a sphere's boundary only
    assert (c_ell > 0).mean() > (c_iso > 0).mean()
