"""Pins of the two-dimensional oracle (Sec. 3 in 2D, App. A, App. B, Eq. radiusAniso2D)
against finite differences, an independent angle definition, closed forms, an
independent numpy estimator and brute-force ray casting."""
import math

import numpy as np
import pytest

import oracle.world2d as O2
from workloads import flat
from workloads.configs import RecordParams

F32 = lambda v: float(np.float32(v))


def fd_grad_hess(fun, x, h=1e-6, hh=1e-4):
    """Central differences: step h for the gradient, hh for the Hessian."""
    x = np.asarray(x, np.float64)
    g = np.zeros(2)
    H = np.zeros((2, 2))
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        g[i] = (fun(x + e) - fun(x - e)) / (2 * h)
        e[i] = hh
        for j in range(2):
            f_ = np.zeros(2)
            f_[j] = hh
            H[i, j] = (fun(x + e + f_) - fun(x + e - f_) - fun(x - e + f_) + fun(x - e - f_)) / (4 * hh * hh)
    return g, H


def test_segment_angle_is_the_signed_subtended_angle():
    rng = np.random.default_rng(0)
    for _ in range(500):
        x, y0, y1 = rng.uniform(0, 1, (3, 2))
        th, g, h, ok = O2.segment_angle(x, y0, y1)
        u, v = y0 - x, y1 - x
        ref = math.atan2(u[0] * v[1] - u[1] * v[0], u @ v)     # independent definition
        assert ok and th == pytest.approx(ref, abs=1e-12)
        th2, g2, h2, _ = O2.segment_angle(x, y1, y0)             # reversed cell: opposite sign
        assert th2 == pytest.approx(-th, abs=1e-12)
        assert np.allclose(g2, -g) and np.allclose(h2, -h)


def test_segment_angle_derivatives_match_finite_differences():
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y0, y1 = rng.uniform(0, 1, (3, 2))
        th, g, h, ok = O2.segment_angle(x, y0, y1)
        if not ok or abs(th) < 0.05 or abs(abs(th) - math.pi) < 0.05:
            continue
        r = min(np.linalg.norm(y0 - x), np.linalg.norm(y1 - x))     # steps scaled to the nearer end
        gf, Hf = fd_grad_hess(lambda p: O2.segment_angle(p, y0, y1)[0], x, h=1e-6 * r, hh=1e-4 * r)
        Hm = np.array([[h[0], h[1]], [h[1], h[2]]])
        scale = max(1.0, np.abs(Hf).max())
        assert np.allclose(g, gf, rtol=1e-7, atol=1e-7 * max(1.0, np.abs(gf).max()))
        assert np.allclose(Hm, Hf, rtol=1e-5, atol=1e-5 * scale)
        assert abs(h[0] + h[2]) <= 1e-9 * scale          # the angle is harmonic in the plane


def test_closed_shell_sums_to_two_pi_with_vanishing_derivatives():
    rng = np.random.default_rng(2)
    x = np.array([0.5, 0.5])
    for n in (4, 7, 64):
        # one vertex per sector (gaps below pi: the polygon surrounds x)
        ang = (np.arange(n) + 0.25 + 0.5 * rng.uniform(size=n)) * 2 * np.pi / n
        r = rng.uniform(0.1, 0.45, n)
        y = x + np.stack([r * np.cos(ang), r * np.sin(ang)], 1)
        tot, gs, hs = 0.0, np.zeros(2), np.zeros(3)
        for j in range(n):
            th, g, h, ok = O2.segment_angle(x, y[j], y[(j + 1) % n])
            tot += th
            gs += g
            hs += h
        assert tot == pytest.approx(2 * np.pi, abs=1e-12)
        assert np.abs(gs).max() < 1e-9 and np.abs(hs).max() < 1e-8


def test_transmittance_derivatives():
    rng = np.random.default_rng(3)
    for _ in range(100):
        x, y = rng.uniform(0, 1, (2, 2))
        st = rng.uniform(0.2, 3)
        T, g, h = O2.transmittance(x, y, st)
        assert T == pytest.approx(math.exp(-st * np.linalg.norm(x - y)), rel=1e-14)
        r = np.linalg.norm(x - y)
        gf, Hf = fd_grad_hess(lambda p: O2.transmittance(p, y, st)[0], x, h=1e-6 * r, hh=1e-4 * r)
        scale = max(1.0, np.abs(Hf).max())
        assert np.allclose(g, gf, rtol=1e-7, atol=1e-9)
        assert np.allclose([h[0], h[1], h[2]], [Hf[0, 0], Hf[0, 1], Hf[1, 1]], rtol=1e-5, atol=1e-5 * scale)


def circle_quadrature(p, R0, st, L0, n=4000):
    """L(p) = (1/2pi) int L0 exp(-st d(theta)) dtheta, p = (px, 0) from the centre."""
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    d = -p * np.cos(th) + np.sqrt(R0 * R0 - p * p * np.sin(th) ** 2)
    return L0 * np.mean(np.exp(-st * d))


def test_constant_radiance_circle():
    R0, L0 = F32(0.3), 1.0
    st = F32(0.8) + F32(0.2)                       # the oracle reads float32 coefficients
    c = O2.OracleScene2(circle=((0.5, 0.5), 0.3, (L0, L0, L0)), sigma_s=0.8, sigma_a=0.2)
    centre = np.array([[0.5, 0.5]], np.float32)
    errs = []
    for N in (64, 256, 1024):
        r = O2.records(c, RecordParams(n_bands=1, n_bins=N, dt=10.0), centre)
        # at the centre: every vertex at R0, angles sum to 2 pi -> L_ff = L0 exp(-st R0)
        assert r["L_ff"][0, 0] == pytest.approx(L0 * math.exp(-st * R0), rel=1e-12)
        assert r["L"][0, 0] == pytest.approx(L0 * math.exp(-st * R0), rel=1e-12)
        assert np.abs(r["grad"][0, 0]).max() < 1e-3
        href = L0 * math.exp(-st * R0) * (st * st / 2 + st / (2 * R0))
        errs.append(abs(r["hess"][0, 0, 0] - href) / href)
        assert abs(r["hess"][0, 0, 1]) < 1e-3 * href
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4
    # off centre: compare with the quadrature (value, and derivatives by FD of it)
    p = 0.12
    pos = np.array([[0.5 + p, 0.5]], np.float32)
    pf = float(pos[0, 0]) - 0.5
    h = 1e-4
    Lq = circle_quadrature(pf, R0, st, L0)
    dL = (circle_quadrature(pf + h, R0, st, L0) - circle_quadrature(pf - h, R0, st, L0)) / (2 * h)
    prev = None
    for N in (128, 512, 2048):
        r = O2.records(c, RecordParams(n_bands=1, n_bins=N, dt=10.0), pos)
        assert r["L"][0, 0] == pytest.approx(Lq, rel=1e-3)
        e = abs(r["grad"][0, 0, 0] - dL) / abs(dL)
        if prev is not None:
            assert e < prev
        prev = e
    assert prev < 0.02


def test_mc_radiance_in_an_empty_square_matches_numpy():
    sc = flat.Scene2(segs=np.zeros((0, 4), np.float32), albedo=np.zeros((0, 3), np.float32), sigma_s=0.8,
                     sigma_a=0.2, lights=[flat.Light2((0.5, 0.92), (1.0, 0.9, 0.8))])
    rp = RecordParams(n_bands=1, n_bins=64, dt=0.1)
    x = np.array([0.31, 0.44], np.float32)
    r = O2.records(O2.OracleScene2(sc), rp, x[None], rec_ids=[5])
    d = O2.ray_directions(rp, rec=5)
    st = F32(0.8) + F32(0.2)
    ss = F32(0.8)
    xd = x.astype(np.float64)
    light = np.array([F32(0.5), F32(0.92)])
    I = np.array([1.0, F32(0.9), F32(0.8)])
    L = np.zeros(3)
    for j in range(64):
        with np.errstate(divide="ignore"):
            t1 = np.where(d[j] > 0, (1 - xd) / d[j], np.where(d[j] < 0, -xd / d[j], np.inf))
        te = t1.min()
        k = 1
        while (k - 0.5) * 0.1 < te:
            t = (k - 0.5) * 0.1
            y = xd + t * d[j]
            dist = np.linalg.norm(light - y)
            Lo = I * math.exp(-st * dist) / (2 * np.pi * dist)
            L += (2 * np.pi / 64) / (2 * np.pi) * ss * 0.1 * math.exp(-st * t) * Lo
            k += 1
    assert np.allclose(r["L"][0], L, rtol=1e-12)
    assert np.all(r["L_ss"][0] == 0)


def test_radius_inverts_the_disc_error_integral():
    rng = np.random.default_rng(4)
    for _ in range(50):
        lam = rng.uniform(0.1, 50)
        LY = rng.uniform(0.05, 2)
        R, st, eig = O2.radius(LY, [lam, 0.0, lam * 0.3], 0.05, 1e-6, 10.0)
        # S.11 in 2D: |lambda| int_disc x_1^2 dA / L over the disc of radius R equals eps
        n = 2000
        rr = (np.arange(n) + 0.5) / n * R
        integral = np.sum(rr ** 3 * (R / n)) * np.pi          # int_0^R r^3 dr * int cos^2
        assert lam * integral / LY == pytest.approx(0.05, rel=1e-5)
        assert np.allclose(eig, np.linalg.eigvalsh([[lam, 0], [0, lam * 0.3]]))


def test_two_by_two_eigenvalues_match_lapack():
    rng = np.random.default_rng(5)
    for _ in range(500):
        h = rng.normal(size=3) * 10 ** rng.uniform(-3, 3)
        _, _, lam = O2.radius(1.0, h, 0.05, 1e-3, 0.5)
        ref = np.linalg.eigvalsh([[h[0], h[1]], [h[1], h[2]]])
        assert np.allclose(lam, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_frozen_record_derivatives_match_finite_differences():
    w = flat.flat_small()
    os_ = O2.OracleScene2(w.scene)
    rp = RecordParams(n_bands=1, n_bins=64)
    for x0 in (np.array([0.2, 0.3], np.float32), np.array([0.8, 0.75], np.float32)):
        base = O2.frozen_eval(os_, rp, x0, 3, x0.astype(np.float64))
        for c in range(3):
            gf, Hf = fd_grad_hess(lambda p: O2.frozen_eval(os_, rp, x0, 3, p)["L_ff"][c], x0.astype(np.float64))
            g = base["grad"][c]
            H = np.array([[base["hess"][c, 0], base["hess"][c, 1]], [base["hess"][c, 1], base["hess"][c, 2]]])
            assert np.allclose(g, gf, rtol=1e-6, atol=1e-8 * max(1, np.abs(gf).max()))
            assert np.allclose(H, Hf, rtol=1e-4, atol=1e-4 * max(1e-3, np.abs(Hf).max()))


def test_trace_matches_numpy_brute_force():
    w = flat.flat_mid()
    os_ = O2.OracleScene2(w.scene)
    rng = np.random.default_rng(6)
    o = w.positions(300, seed=9).astype(np.float64)
    a = rng.uniform(0, 2 * np.pi, 300)
    d = np.stack([np.cos(a), np.sin(a)], 1)
    ids, t = O2.trace(os_, o, d)
    S = w.scene.segs.astype(np.float64)
    for i in range(300):
        best, bt = -1, np.inf
        for k in range(S.shape[0]):
            p0, e = S[k, :2], S[k, 2:] - S[k, :2]
            M = np.array([[d[i, 0], -e[0]], [d[i, 1], -e[1]]])
            if abs(np.linalg.det(M)) < 1e-15:
                continue
            tt, u = np.linalg.solve(M, p0 - o[i])
            if tt > 1e-6 and 0 <= u <= 1 and tt < bt:
                best, bt = k, tt
        assert ids[i] == best
        if best >= 0:
            assert t[i] == pytest.approx(bt, rel=1e-12)


def test_replaying_own_hits_changes_nothing():
    """Replay mode of the 2D oracle: given its own primary hit segments, a record is
    unchanged; given a miss for one ray that hits, only that ray's terms change (its
    surface radiance leaves the Monte Carlo sum, its shells run to the square's edge)."""
    w = flat.flat_small()
    pos = w.positions(16)
    osc = O2.OracleScene2(w.scene)
    r = O2.records(osc, w.params, pos)
    N = w.params.n_bins
    dirs = np.stack([O2.ray_directions(w.params, i) for i in range(pos.shape[0])])
    hits = np.stack([O2.trace(osc, np.repeat(pos[i:i + 1].astype(np.float64), N, 0), dirs[i])[0]
                     for i in range(pos.shape[0])]).astype(np.int32)
    rr = O2.records(osc, w.params, pos, replay_hits=hits)
    for k in ("L", "grad", "hess", "radius"):
        assert np.array_equal(rr[k], r[k]), k
    assert np.all(rr["prim_near"] == 0)
    h2 = hits.copy()
    j = int(np.flatnonzero(hits[0] >= 0)[0])
    h2[0, j] = -1
    r2 = O2.records(osc, w.params, pos[:1], replay_hits=h2[:1])
    assert not np.array_equal(r2["L_ss"][0], r["L_ss"][0])
    assert np.all(r2["L_ss"][0] < r["L_ss"][0] + 1e-15)
