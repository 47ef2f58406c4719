"""Pins of the oracle's ellipsoidal records (Eq. radiusAniso3D per eigenvalue; the query's
ellipsoidal distance ratio) against LAPACK, constructed matrices with known eigenpairs,
the isotropic radius (itself pinned by the ball integral) and the isotropic query."""
import numpy as np
import pytest

import oracle as O

EPS, RMIN, RMAX = 0.05, 1e-3, 0.5


def rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def sym6(H):
    return np.array([H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])


def random_spectrum(rng, kind):
    if kind == "distinct":
        return rng.normal(0, 3, 3)
    if kind == "double":
        a, b = rng.normal(0, 3, 2)
        return np.array([a, a, b])
    if kind == "triple":
        return np.full(3, rng.normal(0, 3))
    if kind == "zero":
        return np.array([0.0, rng.normal(0, 3), rng.normal(0, 3)])
    if kind == "near":
        a = rng.normal(0, 3)
        return np.array([a, a * (1 + 1e-9), rng.normal(0, 3)])
    raise ValueError(kind)


def test_eigenpairs_match_lapack():
    rng = np.random.default_rng(0)
    for kind in ("distinct", "double", "triple", "zero", "near"):
        for _ in range(400):
            Q = rotation(rng)
            H = Q @ np.diag(random_spectrum(rng, kind)) @ Q.T
            H = 0.5 * (H + H.T)
            lam, _, axes, _, _ = O.aniso(1.0, sym6(H), EPS, RMIN, RMAX)
            ref = np.linalg.eigvalsh(H)
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.allclose(lam, ref, rtol=0, atol=1e-12 * scale), (kind, lam, ref)
            # each row is a unit eigenvector of its eigenvalue, and the rows are orthonormal
            assert np.allclose(axes @ axes.T, np.eye(3), atol=1e-12)
            for i in range(3):
                assert np.linalg.norm(H @ axes[i] - lam[i] * axes[i]) <= 1e-11 * scale
            if kind == "distinct":
                w, V = np.linalg.eigh(H)
                for i in range(3):   # projectors are unique when the eigenvalues are
                    assert np.allclose(np.outer(axes[i], axes[i]), np.outer(V[:, i], V[:, i]), atol=1e-9)


def test_radii_follow_each_eigenvalue_along_its_axis():
    rng = np.random.default_rng(1)
    for _ in range(300):
        Q = rotation(rng)
        lam = rng.normal(0, 1, 3) * 10.0 ** rng.uniform(-2, 2, 3)
        H = Q @ np.diag(lam) @ Q.T
        LY = float(rng.uniform(0.01, 2.0))
        lam_o, radii, axes, metric, st = O.aniso(LY, sym6(H), EPS, RMIN, RMAX)
        # the radius of an axis is the isotropic radius of a Hessian |lambda_i| I
        iso = np.array([O.radius(LY, sym6(abs(l) * np.eye(3)), EPS, RMIN, RMAX)[0] for l in np.sort(lam)])
        assert np.allclose(radii, iso, rtol=1e-12)
        # the region's matrix built from the constructed eigenpairs
        order = np.argsort(lam)
        M = sum(np.outer(Q[:, j], Q[:, j]) / iso[i] ** 2 for i, j in enumerate(order))
        assert np.allclose(O.metric_matrix(metric), M, rtol=1e-10, atol=1e-10 * np.abs(M).max())
        # the smallest principal radius is the isotropic record's radius (largest |lambda|)
        R_iso = O.radius(LY, sym6(H), EPS, RMIN, RMAX)[0]
        assert abs(radii.min() - R_iso) <= 1e-12 * R_iso


def test_isotropic_hessian_gives_a_sphere():
    for lam in (-3.0, 0.7, 25.0):
        _, radii, _, metric, _ = O.aniso(0.4, sym6(lam * np.eye(3)), EPS, RMIN, RMAX)
        R = O.radius(0.4, sym6(lam * np.eye(3)), EPS, RMIN, RMAX)[0]
        assert np.allclose(radii, R, rtol=1e-14)
        assert np.allclose(O.metric_matrix(metric), np.eye(3) / R ** 2, rtol=1e-12)


def test_clamps_and_status():
    H = sym6(np.diag([0.0, 1e-12, 1e6]))
    _, radii, _, _, st = O.aniso(1.0, H, EPS, RMIN, RMAX)
    assert radii[0] == RMAX and radii[1] == RMAX       # zero and tiny eigenvalues: r_max
    assert radii[2] == pytest.approx((15 * EPS / (4 * np.pi * 1e6)) ** 0.2, rel=1e-12)
    assert st & 4                                       # CLAMP_HI bit
    _, radii, _, _, st = O.aniso(-1.0, H, EPS, RMIN, RMAX)
    assert np.all(radii == RMIN) and st & 2             # non-positive luminance: r_min
    _, radii, _, _, st = O.aniso(float("nan"), H, EPS, RMIN, RMAX)
    assert np.all(radii == RMIN) and st & 1


def synthetic_ellipsoids(rng, n, kind="aniso"):
    pos = rng.uniform(0.2, 0.8, (n, 3))
    metric = np.zeros((n, 6))
    frames = np.zeros((n, 3, 3))
    radii = np.zeros((n, 3))
    for k in range(n):
        Q = rotation(rng)
        r = rng.uniform(0.05, 0.3, 3) if kind == "aniso" else np.full(3, rng.uniform(0.05, 0.3))
        frames[k], radii[k] = Q, r
        metric[k] = sym6(Q @ np.diag(1.0 / r ** 2) @ Q.T)
    return pos, metric, frames, radii


def test_query_with_spheres_equals_isotropic_query():
    rng = np.random.default_rng(2)
    n = 60
    pos = rng.uniform(0.2, 0.8, (n, 3))
    R = rng.uniform(0.05, 0.3, n)
    L, grad, hess = rng.normal(size=(n, 3)), rng.normal(size=(n, 9)), rng.normal(size=(n, 18))
    metric = np.stack([sym6(np.eye(3) / r ** 2) for r in R])
    q = rng.uniform(0, 1, (500, 3))
    for order in (1, 2):
        a, ca, _ = O.query(pos, R, L, grad, hess, q, order)
        b, cb, _ = O.query_aniso(pos, metric, L, grad, hess, q, order)
        assert np.array_equal(ca, cb)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_query_membership_along_principal_axes():
    rng = np.random.default_rng(3)
    pos, metric, frames, radii = synthetic_ellipsoids(rng, 1)
    L, grad = np.ones((1, 3)), np.zeros((1, 9))
    for i in range(3):
        for s in (-1, 1):
            inside = pos[0] + s * (1 - 1e-6) * radii[0, i] * frames[0][:, i]
            outside = pos[0] + s * (1 + 1e-6) * radii[0, i] * frames[0][:, i]
            _, c_in, _ = O.query_aniso(pos, metric, L, grad, None, inside[None])
            _, c_out, _ = O.query_aniso(pos, metric, L, grad, None, outside[None])
            assert c_in[0] == 1 and c_out[0] == 0


def test_query_membership_matches_frame_coordinates():
    # membership by the record frame: |diag(1/R) Q^T D| < 1, computed without the metric
    rng = np.random.default_rng(4)
    pos, metric, frames, radii = synthetic_ellipsoids(rng, 40)
    L, grad = np.ones((40, 3)), np.zeros((40, 9))
    q = rng.uniform(0, 1, (2000, 3))
    _, cnt, near = O.query_aniso(pos, metric, L, grad, None, q)
    D = q[:, None, :] - pos[None, :, :]
    u = np.einsum("kij,qki->qkj", frames, D) / radii[None]
    ref = (np.linalg.norm(u, axis=2) < 1.0).sum(axis=1)
    ok = near.astype(bool) | (cnt == ref)
    assert ok.all() and near.mean() < 0.01


def test_query_reproduces_linear_and_quadratic_fields():
    rng = np.random.default_rng(5)
    n = 80
    pos, metric, _, _ = synthetic_ellipsoids(rng, n)
    a0, b = rng.normal(size=3), rng.normal(size=(3, 3))
    Hq = [(lambda A: A + A.T)(rng.normal(size=(3, 3))) for _ in range(3)]
    q = rng.uniform(0.3, 0.7, (400, 3))
    # linear field L_c(x) = a0_c + b_c . x with exact gradients: reproduced at order 1
    L = a0[None] + pos @ b.T
    grad = np.repeat(b.reshape(1, 9), n, axis=0)
    out, cnt, _ = O.query_aniso(pos, metric, L, grad, None, q, 1)
    hit = cnt > 0
    assert hit.mean() > 0.5
    assert np.allclose(out[hit], a0[None] + q[hit] @ b.T, atol=1e-12)
    # quadratic field with exact gradients and Hessians: reproduced at order 2
    Lq = np.stack([a0[c] + pos @ b[c] + 0.5 * np.einsum("ki,ij,kj->k", pos, Hq[c], pos) for c in range(3)], 1)
    gq = np.concatenate([b[c][None] + pos @ Hq[c] for c in range(3)], axis=1)
    hq = np.concatenate([np.repeat(sym6(Hq[c])[None], n, 0) for c in range(3)], axis=1)
    out, cnt, _ = O.query_aniso(pos, metric, Lq, gq, hq, q, 2)
    ref = np.stack([a0[c] + q @ b[c] + 0.5 * np.einsum("ki,ij,kj->k", q, Hq[c], q) for c in range(3)], 1)
    assert np.allclose(out[hit], ref[hit], atol=1e-11)


def test_query_weights_from_record_frames():
    # two overlapping records with constant radiance 1 and 3: the result is the weighted
    # mean with w = 3d^2 - 2d^3, d = 1 - |diag(1/R) Q^T D| computed from the frames
    rng = np.random.default_rng(6)
    pos, metric, frames, radii = synthetic_ellipsoids(rng, 2)
    pos[1] = pos[0] + 0.3 * radii[0, 0] * frames[0][:, 0]
    L = np.array([[1.0, 1.0, 1.0], [3.0, 3.0, 3.0]])
    grad = np.zeros((2, 9))
    checked = 0
    for delta in (0.5, 1e-1, 1e-2, 1e-3):
        x = pos[1] + (1 - delta) * radii[1, 2] * frames[1][:, 2]
        w = []
        for k in range(2):
            rho = np.linalg.norm((frames[k].T @ (x - pos[k])) / radii[k])
            d = 1.0 - rho
            w.append(3 * d * d - 2 * d ** 3 if rho < 1 else 0.0)
        out, cnt, _ = O.query_aniso(pos, metric, L, grad, None, x[None])
        assert cnt[0] == sum(wk > 0 for wk in w)
        if cnt[0]:
            assert out[0, 0] == pytest.approx((w[0] + 3 * w[1]) / (w[0] + w[1]), rel=1e-12)
            checked += 1
    assert checked >= 3
