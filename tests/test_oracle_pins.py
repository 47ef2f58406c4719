"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, closed forms (octant solid angle, constant-radiance sphere,
ball integral), finite differences of the oracle's own value functions (which
test its closed-form derivatives, App. A and App. C), brute force (Monte Carlo
solid angle, all-triangle ray casting, independent numpy geometry), and
invariants (closed shells sum to 4 pi, symmetric Hessians, partition of unity).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.configs import RecordParams
from workloads.scenes import Medium, PointLight, Scene, cube_walls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
rng0 = np.random.default_rng(12345)


def fd_grad(f, x, h=1e-6):
    return np.array([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(3)])


def fd_hess_from_grad(g, x, h=1e-6):
    """Hessian by central differences of an analytic gradient function."""
    return np.stack([(g(x + h * e) - g(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)


def fd_hess(f, x, h=1e-4):
    H = np.zeros((3, 3))
    E = np.eye(3) * h
    for i in range(3):
        for j in range(3):
            H[i, j] = (f(x + E[i] + E[j]) - f(x + E[i] - E[j]) - f(x - E[i] + E[j]) + f(x - E[i] - E[j])) / (4 * h * h)
    return H


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------- generator
def test_splitmix64_published_outputs(oracle_lib):
    gamma = 0x9E3779B97F4A7C15
    path = os.path.join(ROOT, "tests", "golden", "splitmix64_seed0.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for k, out in rows:
        assert O.splitmix64((int(k) * gamma) % (1 << 64)) == int(out, 16)


def test_jitter_uniform_on_24bit_grid(oracle_lib):
    u = np.array([O.jitter(3, r, i, j, s) for r in range(4) for i in range(16) for j in range(32) for s in range(2)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))          # exact 24-bit values
    assert len(np.unique(u)) > 0.99 * len(u)
    # Kolmogorov-Smirnov against U[0,1): D < 1.63/sqrt(n) at 1% level
    us = np.sort(u)
    n = len(us)
    D = max(np.max(np.arange(1, n + 1) / n - us), np.max(us - np.arange(n) / n))
    assert D < 1.63 / math.sqrt(n)


# ----------------------------------------------------------------- ray set
def test_ray_directions_lie_in_equal_solid_angle_strata(oracle_lib):
    rp = RecordParams(n_bands=8, n_bins=16)
    d = O.ray_directions(rp, rec=7)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    N = 8 * 16
    assert np.allclose(d[N], [0, 0, 1]) and np.allclose(d[N + 1], [0, 0, -1])
    for v in range(N):
        i, j = divmod(v, 16)
        ct = d[v, 2]
        assert 1 - 2 * (i + 1) / 8 <= ct <= 1 - 2 * i / 8
        ph = math.atan2(d[v, 1], d[v, 0]) % (2 * math.pi)
        assert 2 * math.pi * j / 16 - 1e-12 <= ph <= 2 * math.pi * (j + 1) / 16 + 1e-12
    # stratum solid angle (d cos theta)(d phi) = (2/Nb)(2 pi/Ns) = 4 pi / N for every stratum
    assert abs(8 * 16 * (2 / 8) * (2 * math.pi / 16) - 4 * math.pi) < 1e-12


def test_cell_topology_is_a_closed_consistently_wound_sphere(oracle_lib):
    for nb, ns in [(2, 3), (8, 16), (5, 7)]:
        cells = O.cell_vertices(nb, ns)
        V, F = nb * ns + 2, cells.shape[0]
        assert F == 2 * V - 4                                     # Euler: V - E + F = 2 with E = 3F/2
        directed = {}
        for a, b, c in cells:
            for e in [(a, b), (b, c), (c, a)]:
                assert e not in directed
                directed[e] = 1
        for (a, b) in directed:
            assert (b, a) in directed                             # every edge used once each way


def test_shell_solid_angles_sum_to_4pi(oracle_lib):
    """Signed Omega over any star-shaped shell of the triangulation is 4 pi (reading R5)."""
    rp = RecordParams(n_bands=8, n_bins=16)
    d = O.ray_directions(rp, rec=3)
    cells = O.cell_vertices(8, 16)
    for trial in range(3):
        rad = rng0.uniform(0.2, 2.0, size=d.shape[0])
        y = d * rad[:, None]
        x = np.zeros(3)
        tot, g, H = 0.0, np.zeros(3), np.zeros((3, 3))
        for a, b, c in cells:
            F, gF, HF, ok = O.formfactor(x, y[a], y[b], y[c], 1)
            tot += F
            g += gF
            H += HF
        assert abs(tot * 4 * math.pi - 4 * math.pi) < 1e-12
        assert np.abs(g).max() < 1e-11 and np.abs(H).max() < 1e-10   # closed shell: sum grad = sum H = 0


# ----------------------------------------------------------------- App. C
def test_solid_angle_octant_closed_form(oracle_lib):
    F, g, H, ok = O.formfactor([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1])
    assert abs(F * 4 * math.pi - math.pi / 2) < 1e-15
    # by symmetry grad F is along (1,1,1): moving toward the face enlarges it
    assert np.allclose(g / np.linalg.norm(g), np.ones(3) / math.sqrt(3), atol=1e-14)


def _mc_solid_angle(x, tri, n, rng):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    a, b, c = tri
    e1, e2 = b - a, c - a
    p = np.cross(d, e2)
    det = p @ e1
    s = x - a
    u = (p @ s) / det
    q = np.cross(s, e1)
    v = (d @ q) / det
    t = (q @ e2) / det
    hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    return 4 * math.pi * hit.mean()


def test_solid_angle_vs_brute_force_monte_carlo(oracle_lib):
    rng = np.random.default_rng(7)
    for trial in range(3):
        x = np.zeros(3)
        tri = [np.array([0.0, 0.0, 1.0]) + rng.normal(size=3) * 0.6 for _ in range(3)]
        F, *_ = O.formfactor(x, *tri, ff_signed=0)
        om = F * 4 * math.pi
        n = 2_000_000
        est = _mc_solid_angle(x, tri, n, rng)
        sd = math.sqrt(om * (4 * math.pi - om) / n)
        assert abs(est - om) < 5 * sd + 1e-9


def test_small_far_triangle_is_projected_area_over_r2(oracle_lib):
    x = np.zeros(3)
    c = np.array([0.3, -0.2, 5.0])
    a = 1e-3
    tri = [c, c + np.array([a, 0, 0.2 * a]), c + np.array([0, a, 0])]
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    area_cos = 0.5 * abs(n @ (c - x)) / np.linalg.norm(c - x)
    F, *_ = O.formfactor(x, *tri, ff_signed=0)
    assert rel(F * 4 * math.pi, area_cos / np.linalg.norm(c) ** 2) < 1e-3


def _random_cell(rng):
    x = rng.normal(size=3) * 0.05
    return x, [x + np.array([0, 0, 1.0]) + rng.normal(size=3) * 0.4 for _ in range(3)]


def test_formfactor_derivatives_vs_finite_differences(oracle_lib):
    rng = np.random.default_rng(1)
    for trial in range(40):
        x, ys = _random_cell(rng)
        for signed in (1, 0):
            F, g, H, ok = O.formfactor(x, *ys, signed)
            f = lambda xx: O.formfactor(xx, *ys, signed)[0]
            assert rel(g, fd_grad(f, x)) < 1e-7
            assert rel(H, fd_hess_from_grad(lambda xx: O.formfactor(xx, *ys, signed)[1], x)) < 1e-7
            assert rel(H, fd_hess(f, x)) < 1e-4
            assert np.linalg.norm(H - H.T) <= 1e-12 * np.linalg.norm(H)   # the printed form is symmetric


def test_printed_grad_A_disagrees_and_corrected_one_agrees():
    """Reading R3: App. C's printed grad A misses a transpose; -(y2-y1)x(y3-y1) is right."""
    rng = np.random.default_rng(2)
    x, ys = _random_cell(rng)
    A = lambda xx: np.dot(ys[0] - xx, np.cross(ys[1] - xx, ys[2] - xx))
    fd = fd_grad(A, x)
    r1, r2, r3 = (y - x for y in ys)
    printed = np.cross(r3 - r2, r1) - np.cross(r2, r3)
    corrected = -np.cross(ys[1] - ys[0], ys[2] - ys[0])
    assert rel(corrected, fd) < 1e-8
    assert rel(printed, fd) > 1e-2


def test_signed_and_absolute_A_agree_on_positive_cells_and_differ_on_folds(oracle_lib):
    x = np.zeros(3)
    pos_tri = [np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])]
    a = O.formfactor(x, *pos_tri, 1)
    b = O.formfactor(x, *pos_tri, 0)
    assert a[0] == b[0] and np.allclose(a[1], b[1]) and np.allclose(a[2], b[2])
    neg = [pos_tri[0], pos_tri[2], pos_tri[1]]
    a = O.formfactor(x, *neg, 1)
    b = O.formfactor(x, *neg, 0)
    assert abs(a[0] + b[0]) < 1e-15 and a[0] < 0


# ----------------------------------------------------------------- App. A, phase
def test_transmittance_closed_form_and_derivatives(oracle_lib):
    rng = np.random.default_rng(3)
    for trial in range(20):
        x, y = rng.normal(size=3) * 0.3, rng.normal(size=3)
        st = rng.uniform(0.1, 3)
        T, g, H = O.transmittance(x, y, st)
        assert abs(T - math.exp(-st * np.linalg.norm(x - y))) < 1e-15
        f = lambda xx: O.transmittance(xx, y, st)[0]
        assert rel(g, fd_grad(f, x)) < 1e-7
        assert rel(H, fd_hess_from_grad(lambda xx: O.transmittance(xx, y, st)[1], x)) < 1e-7


def test_hg_normalised_with_mean_cosine_g(oracle_lib):
    mu, w = np.polynomial.legendre.leggauss(400)
    for g in (0.0, 0.3, 0.7, -0.5):
        f = np.array([O.hg(m, g) for m in mu])
        assert abs(2 * math.pi * np.sum(w * f) - 1.0) < 1e-10
        assert abs(2 * math.pi * np.sum(w * f * mu) - g) < 1e-10
    assert abs(O.hg(0.3, 0.0) - 1 / (4 * math.pi)) < 1e-16


def test_phase_derivatives_vs_finite_differences(oracle_lib):
    rng = np.random.default_rng(4)
    for trial in range(20):
        x, y = rng.normal(size=3) * 0.3, rng.normal(size=3)
        wo = rng.normal(size=3)
        wo /= np.linalg.norm(wo)
        g = rng.uniform(-0.8, 0.8)
        v, gr, H = O.phase(x, y, wo, g)
        wi = (x - y) / np.linalg.norm(x - y)
        assert abs(v - O.hg(wi @ wo, g)) < 1e-15
        f = lambda xx: O.phase(xx, y, wo, g)[0]
        assert rel(gr, fd_grad(f, x)) < 1e-7
        assert rel(H, fd_hess_from_grad(lambda xx: O.phase(xx, y, wo, g)[1], x)) < 1e-7


# ----------------------------------------------------------------- Sec. 4 cell algebra
def test_cell_derivatives_vs_finite_differences(oracle_lib):
    rng = np.random.default_rng(5)
    Lo = np.array([0.3, 0.2, 0.1])
    for trial in range(30):
        x, ys = _random_cell(rng)
        l = int(np.argmax([np.linalg.norm(y - x) for y in ys]))
        args = (l, Lo, 1.2, 0.6, [0, 0.6, 0.8], 0.7)
        L, g, H, ok = O.cell(x, *ys, *args)
        for c in range(3):
            f = lambda xx: O.cell(xx, *ys, *args)[0][c]
            assert rel(g[c], fd_grad(f, x)) < 1e-7
            assert rel(H[c], fd_hess_from_grad(lambda xx: O.cell(xx, *ys, *args)[1][c], x)) < 1e-7
            assert np.linalg.norm(H[c] - H[c].T) <= 1e-12 * np.linalg.norm(H[c])
        assert np.allclose(L / Lo, L[0] / Lo[0])                 # linear in L_o, channel by channel


def test_cell_with_tied_furthest_vertices_vs_finite_differences(oracle_lib):
    """Reading R9: tied furthest vertices average their reduced radiance; still exact derivatives."""
    rng = np.random.default_rng(15)
    for trial in range(10):
        x = rng.normal(size=3) * 0.02
        d = rng.normal(size=(3, 3)) * 0.3 + np.array([0, 0, 1.0])
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        ys = [x0 for x0 in 0.35 * d]                             # three vertices at one distance
        Lo = rng.uniform(0.1, 1.0, size=(3, 3))
        args = ([0, 1, 2], Lo, 0.9, 0.4, [0.6, 0, 0.8], 0.3)
        L, g, H, ok = O.cell(np.zeros(3), *ys, *args)
        for c in range(3):
            f = lambda xx: O.cell(xx, *ys, *args)[0][c]
            assert rel(g[c], fd_grad(f, np.zeros(3))) < 1e-7
            assert rel(H[c], fd_hess_from_grad(lambda xx: O.cell(xx, *ys, *args)[1][c], np.zeros(3))) < 1e-7
        single = sum(O.cell(np.zeros(3), *ys, q, Lo, 0.9, 0.4, [0.6, 0, 0.8], 0.3)[0] for q in range(3)) / 3
        assert np.allclose(L, single, rtol=1e-13)                # mean of the three single-vertex cells


def test_general_product_rule_reduces_to_simplified_at_g0(oracle_lib):
    """At g = 0 the general Eqs. (grad f = H f = 0) equal the simplified Eqs."""
    rng = np.random.default_rng(6)
    for trial in range(20):
        x, ys = _random_cell(rng)
        a = O.cell(x, *ys, 0, [0.3, 0.2, 0.1], 1.1, 0.0, [0, 0, 1], 0.5, general=1)
        b = O.cell(x, *ys, 0, [0.3, 0.2, 0.1], 1.1, 0.0, [0, 0, 1], 0.5, general=0)
        for u, v in zip(a[:3], b[:3]):
            assert np.allclose(u, v, rtol=1e-13, atol=1e-300)
    c1 = W.config1()
    c1.scene.medium = Medium(0.5, 0.05, 0.0)
    os_ = O.OracleScene(c1.scene)
    pos = c1.positions()[:4]
    ra = O.records(os_, c1.params, pos, general_derivs=1)
    rb = O.records(os_, c1.params, pos, general_derivs=0)
    for k in ("L", "grad", "hess", "L_ff"):
        assert np.allclose(ra[k], rb[k], rtol=1e-12, atol=1e-14)


def test_record_derivatives_vs_frozen_vertex_finite_differences(oracle_lib):
    """P3: grad and Hessian of the record equal FD of its own L_ff with the shells frozen."""
    c1 = W.config1()
    os_ = O.OracleScene(c1.scene)
    pos = c1.positions()
    for r in (0, 5, 11):
        x0 = pos[r].astype(np.float64)
        for which in (1, 2):
            fL = lambda xx: O.frozen_eval(os_, c1.params, pos[r], xx, rec=r, which=which)[0][0]
            fg = lambda xx: O.frozen_eval(os_, c1.params, pos[r], xx, rec=r, which=which)[1][0]
            L, g, H = O.frozen_eval(os_, c1.params, pos[r], x0, rec=r, which=which)
            for c in range(3):
                assert rel(g[0, c], fd_grad(lambda xx: fL(xx)[c], x0)) < 1e-6
                assert rel(H[0, c], fd_hess_from_grad(lambda xx: fg(xx)[c], x0)) < 1e-6
        rec = O.records(os_, c1.params, pos[r:r + 1], rec_ids=[r])
        L, g, H = O.frozen_eval(os_, c1.params, pos[r], x0, rec=r, which=0)
        assert np.allclose(rec["grad"][0].reshape(3, 3), g[0], rtol=1e-12, atol=1e-14)
        assert np.allclose(rec["L_ff"][0], L[0], rtol=1e-12)
        h6 = rec["hess"][0].reshape(3, 6)
        for c in range(3):
            Hf = H[0, c]
            assert np.allclose(h6[c], [Hf[0, 0], Hf[0, 1], Hf[0, 2], Hf[1, 1], Hf[1, 2], Hf[2, 2]], rtol=1e-12,
                               atol=1e-12)
            assert np.linalg.norm(Hf - Hf.T) <= 1e-12 * np.linalg.norm(Hf)   # P5


# ----------------------------------------------------------------- P6 closed form
def _sphere_L(p, R0, st, L0=1.0, n=200):
    mu, w = np.polynomial.legendre.leggauss(n)
    s = np.sqrt(R0 * R0 - p * p * (1 - mu * mu))
    d = -p * mu + s
    d1 = -mu - p * (1 - mu * mu) / s
    d2 = -(1 - mu * mu) / s - p * p * (1 - mu * mu) ** 2 / s ** 3
    e = np.exp(-st * d)
    L = 0.5 * L0 * np.sum(w * e)
    L1 = 0.5 * L0 * np.sum(w * (-st * d1) * e)
    L2 = 0.5 * L0 * np.sum(w * (st * st * d1 * d1 - st * d2) * e)
    return L, L1, L2


def test_sphere_quadrature_matches_centre_closed_form():
    R0, st = 0.4, 1.5
    L, L1, L2 = _sphere_L(1e-9, R0, st)
    e = math.exp(-st * R0)
    assert abs(L - e) < 1e-14
    assert abs(L2 - e * (st * st / 3 + 2 * st / (3 * R0))) < 1e-10


@pytest.mark.parametrize("g", [0.0, 0.5])
def test_constant_radiance_sphere_centre(oracle_lib, g):
    """At the centre: L = L0 e^{-st R0}, grad L = -g st L ω_o, H L = L[st/R0 (I-M) + st^2 M],
    M = (1-g^2)/3 I + g^2 ω_o ω_o^T (HG second moment)."""
    R0, st, c = 0.4, 1.5, np.array([0.5, 0.5, 0.5])
    os_ = O.OracleScene(sphere=dict(center=c, radius=R0, Le=(1.0, 1.0, 1.0), sigma_t=st, g=g))
    R0 = float(np.float32(R0))                  # the oracle reads the radius as float32
    wo = np.array([0.0, 0.0, 1.0])
    e = math.exp(-st * R0)
    M = (1 - g * g) / 3 * np.eye(3) + g * g * np.outer(wo, wo)
    Href = e * (st / R0 * (np.eye(3) - M) + st * st * M)
    gref = -g * st * e * wo
    errs = []
    for nb in (16, 32, 64, 128):
        rp = RecordParams(n_bands=nb, n_bins=2 * nb, omega_o=tuple(wo))
        r = O.records(os_, rp, c[None].astype(np.float32), surface_only=1)
        h = r["hess"][0, :6]
        H = np.array([[h[0], h[1], h[2]], [h[1], h[3], h[4]], [h[2], h[4], h[5]]])
        errs.append((abs(r["L"][0, 0] - e) / e, np.linalg.norm(r["grad"][0, :3] - gref) / (st * e),
                     rel(H, Href)))
    errs = np.array(errs)
    assert errs[-1, 0] < (1e-12 if g == 0 else 1e-4)   # MC: exact at g = 0 (constant integrand)
    assert errs[-1, 1] < 2e-4 and errs[-1, 2] < 3e-3
    assert np.all(np.diff(errs[:, 2]) < 0)              # consistent: converges with the ray count
    assert np.all(np.diff(errs[:, 1]) < 0)


def test_constant_radiance_sphere_off_centre(oracle_lib):
    R0, st, c = 0.4, 1.5, np.array([0.5, 0.5, 0.5])
    os_ = O.OracleScene(sphere=dict(center=c, radius=R0, Le=(1.0, 1.0, 1.0), sigma_t=st, g=0.0))
    R0 = float(np.float32(R0))
    p = 0.15
    phat = np.array([0.6, 0.0, 0.8])
    x = (c + p * phat).astype(np.float32)
    p = float(np.linalg.norm(x.astype(np.float64) - c))
    phat = (x.astype(np.float64) - c) / p
    L, L1, L2 = _sphere_L(p, R0, st)
    gref = L1 * phat
    Href = L2 * np.outer(phat, phat) + (L1 / p) * (np.eye(3) - np.outer(phat, phat))
    errs = []
    for nb in (16, 32, 64, 128):
        rp = RecordParams(n_bands=nb, n_bins=2 * nb)
        r = O.records(os_, rp, x[None], surface_only=1)
        h = r["hess"][0, :6]
        H = np.array([[h[0], h[1], h[2]], [h[1], h[3], h[4]], [h[2], h[4], h[5]]])
        errs.append((abs(r["L"][0, 0] - L) / L, rel(r["grad"][0, :3], gref), rel(H, Href)))
    errs = np.array(errs)
    assert errs[-1, 0] < 1e-5
    # "biased but consistent" (Sec. 4): freezing T at the furthest vertex leaves a bias of
    # first order in the cell size, so the error halves each time the band count doubles
    ratio = errs[1:, 1] / errs[:-1, 1]
    assert np.all((ratio > 0.4) & (ratio < 0.6))
    assert np.all(np.diff(errs[:, 2]) < 0)
    assert errs[-1, 1] < 0.04 and errs[-1, 2] < 0.01


# ----------------------------------------------------------------- MC radiance, convex room
def _room_reference(x, dirs, N, scene, dt):
    """Independent numpy evaluation of Eqs. outLF/mediaLFin/curveLFin along given directions
    in the empty unit-cube room (no occluders: every light path is visible)."""
    m = scene.medium
    st = float(np.float32(m.sigma_s)) + float(np.float32(m.sigma_a))
    ss, g = float(np.float32(m.sigma_s)), float(np.float32(m.g))
    lp = np.array(scene.lights[0].pos, np.float32).astype(np.float64)
    I = np.array(scene.lights[0].intensity, np.float32).astype(np.float64)
    rho = float(np.float32(0.7))
    hg = lambda mu: (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)
    d = dirs[:N]
    with np.errstate(divide="ignore"):
        tpos = np.where(d > 0, (1 - x) / d, np.where(d < 0, -x / d, np.inf))
    axis = np.argmin(tpos, axis=1)
    te = tpos[np.arange(N), axis]
    y = x + te[:, None] * d
    n = np.zeros((N, 3))
    n[np.arange(N), axis] = -np.sign(d[np.arange(N), axis])       # wall normal facing x
    l = lp - y
    dist = np.linalg.norm(l, axis=1)
    cs = np.maximum(0, np.sum(n * l, axis=1) / dist)
    Lsurf = rho / math.pi * I[None] * (cs * np.exp(-st * dist) / dist ** 2)[:, None]
    K = int(math.ceil(te.max() / dt))
    fx = hg(-d @ np.array([0, 0, 1.0]))
    w = 4 * math.pi / N * fx
    Lss = np.sum((w * np.exp(-st * te))[:, None] * Lsurf, axis=0)
    Lms = np.zeros(3)
    for k in range(1, K + 1):
        tk = (k - 0.5) * dt
        yk = x + tk * d
        lk = lp - yk
        dk = np.linalg.norm(lk, axis=1)
        mu = np.sum(lk * d, axis=1) / dk
        Lo = hg(mu)[:, None] * I[None] * (np.exp(-st * dk) / dk ** 2)[:, None]
        on = tk < te
        Lms += np.sum((w * on * ss * dt * math.exp(-st * tk))[:, None] * Lo, axis=0)
    return Lss, Lms


def test_mc_radiance_in_empty_room_matches_independent_evaluation(oracle_lib):
    tris = cube_walls()
    scene = Scene(tris=tris, albedo=np.full((12, 3), 0.7, np.float32), medium=Medium(0.5, 0.05, 0.3),
                  lights=[PointLight((0.5, 0.5, 0.92), (1.0, 0.9, 0.8))])
    os_ = O.OracleScene(scene)
    rp = RecordParams(n_bands=16, n_bins=32)
    pos = np.array([[0.3, 0.4, 0.5], [0.7, 0.2, 0.3], [0.5, 0.5, 0.6]], np.float32)
    r = O.records(os_, rp, pos, rec_ids=[0, 1, 2])
    for k in range(3):
        dirs = O.ray_directions(rp, rec=k)
        Lss, Lms = _room_reference(pos[k].astype(np.float64), dirs, 16 * 32, scene, float(np.float32(0.1)))
        assert np.allclose(r["L_ss"][k], Lss, rtol=1e-10)
        assert np.allclose(r["L_ms"][k], Lms, rtol=1e-10)


# ----------------------------------------------------------------- P7 radius + eigen
def test_radius_inverts_the_ball_integral_of_the_error(oracle_lib):
    """For H = lambda I: |lambda| int_ball x1^2 dV / L = eps at the returned R (Eq. radiusAniso3D)."""
    rng = np.random.default_rng(8)
    r_n, w_r = np.polynomial.legendre.leggauss(40)
    for trial in range(5):
        lam, L, eps = rng.uniform(0.5, 50), rng.uniform(0.01, 2), 0.05
        R, st, _ = O.radius(L, [lam, 0, 0, lam, 0, lam], eps, 1e-9, 1e9)
        # int_ball x1^2 dV = int_0^R r^2 * (int_sphere x1^2 dA at radius r) dr, with the shell
        # integral 4 pi r^4 / 3 evaluated by quadrature in cos(theta)
        mu, wm = np.polynomial.legendre.leggauss(20)
        shell = lambda r: 2 * math.pi * r * r * np.sum(wm * (r * r * (1 - mu * mu) / 2))
        rr = 0.5 * R * (r_n + 1)
        integral = 0.5 * R * np.sum(w_r * np.array([shell(x) for x in rr]))
        assert abs(lam * integral / L - eps) < 1e-12


def test_radius_clamps_and_status(oracle_lib):
    R, st, _ = O.radius(0.5, [0] * 6, 0.05, 1e-3, 0.5)
    assert R == pytest.approx(0.5) and st & 4
    R, st, _ = O.radius(-1.0, [1, 0, 0, 1, 0, 1], 0.05, 1e-3, 0.5)
    assert R == pytest.approx(1e-3) and st & 2
    R, st, _ = O.radius(float("nan"), [1, 0, 0, 1, 0, 1], 0.05, 1e-3, 0.5)
    assert st & 1


def test_jacobi_eigenvalues_vs_lapack(oracle_lib):
    rng = np.random.default_rng(9)
    mats = []
    for t in range(2000):
        A = rng.normal(size=(3, 3))
        mats.append(A + A.T)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    mats += [Q @ np.diag([1.0, 1.0, -2.0]) @ Q.T, Q @ np.diag([0.0, 0.0, 3.0]) @ Q.T, np.zeros((3, 3)),
             np.eye(3) * 4.0, Q @ np.diag([1e-9, 1.0, 1e9]) @ Q.T]
    for M in mats:
        h6 = [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]]
        lam = O.eig3(h6)
        ref = np.linalg.eigvalsh(M)
        assert np.allclose(lam, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))


# ----------------------------------------------------------------- P8 query
def _rand_records(rng, n):
    pos = rng.uniform(0.2, 0.8, size=(n, 3))
    R = rng.uniform(0.05, 0.3, size=n)
    L = rng.uniform(0.1, 1, size=(n, 3))
    g = rng.normal(size=(n, 9))
    h = rng.normal(size=(n, 18))
    return pos, R, L, g, h


def test_query_at_a_record_centre_returns_its_radiance(oracle_lib):
    rng = np.random.default_rng(10)
    pos, R, L, g, h = _rand_records(rng, 1)
    out, st, near = O.query(pos, R, L, g, h, pos)
    assert st[0] == 1 and np.allclose(out[0], L[0], rtol=1e-15)


def test_query_reproduces_linear_and_quadratic_fields(oracle_lib):
    """Partition of unity: records carrying exact derivatives reproduce linear fields
    (order 1) and quadratic fields (order 2) exactly wherever some record covers x'."""
    rng = np.random.default_rng(11)
    n = 40
    pos, R, _, _, _ = _rand_records(rng, n)
    a = rng.normal(size=3)
    b = rng.normal(size=(3, 3))
    Qm = rng.normal(size=(3, 3, 3))
    Qm = Qm + Qm.transpose(0, 2, 1)
    lin = lambda x: a + b @ x
    L = np.array([lin(p) for p in pos])
    g = np.array([b.reshape(-1) for _ in pos])
    q = rng.uniform(0.2, 0.8, size=(500, 3))
    out, st, _ = O.query(pos, R, L, g, None, q, order=1)
    cov = st > 0
    assert cov.sum() > 100
    assert np.allclose(out[cov], np.array([lin(x) for x in q[cov]]), rtol=1e-12, atol=1e-12)
    assert np.all(out[~cov] == 0)
    quad = lambda x: a + b @ x + 0.5 * np.einsum("cij,i,j->c", Qm, x, x)
    L2 = np.array([quad(p) for p in pos])
    g2 = np.array([(b + np.einsum("cij,j->ci", Qm, p)).reshape(-1) for p in pos])
    h2 = np.array([[Qm[c][i, j] for c in range(3) for (i, j) in
                    [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]] for _ in pos])
    out, st, _ = O.query(pos, R, L2, g2, h2, q, order=2)
    assert np.allclose(out[cov], np.array([quad(x) for x in q[cov]]), rtol=1e-11, atol=1e-11)


def test_query_weight_vanishes_continuously_at_the_radius(oracle_lib):
    pos = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5]])
    R = np.array([0.2, 0.2])
    L = np.array([[1.0, 1, 1], [3.0, 3, 3]])
    g = np.zeros((2, 9))
    x_in = np.array([[0.7 - 1e-9, 0.5, 0.5]])
    x_out = np.array([[0.7 + 1e-9, 0.5, 0.5]])
    a, sa, _ = O.query(pos, R, L, g, None, x_in)
    b, sb, _ = O.query(pos, R, L, g, None, x_out)
    assert sa[0] == 2 and sb[0] == 1
    assert np.allclose(a, b, atol=1e-8)


# ----------------------------------------------------------------- P9 traversal
def _numpy_closest(o, d, tris):
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    e1, e2 = b - a, c - a
    out_t = np.full(o.shape[0], np.inf)
    out_i = np.full(o.shape[0], -1)
    for k in range(o.shape[0]):
        p = np.cross(d[k], e2)
        det = np.einsum("ij,ij->i", e1, p)
        with np.errstate(divide="ignore", invalid="ignore"):
            s = o[k] - a
            u = np.einsum("ij,ij->i", s, p) / det
            q = np.cross(s, e1)
            v = (q @ d[k]) / det
            t = np.einsum("ij,ij->i", q, e2) / det
        ok = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-6)
        if ok.any():
            tt = np.where(ok, t, np.inf)
            i = int(np.argmin(tt))
            out_t[k], out_i[k] = tt[i], i
    return out_i, out_t


def test_traversal_bvh_equals_brute_force_and_numpy(oracle_lib):
    c2 = W.config2()
    ob = O.OracleScene(c2.scene, use_bvh=True)
    on = O.OracleScene(c2.scene, use_bvh=False)
    rng = np.random.default_rng(13)
    o = np.repeat(c2.positions()[:20].astype(np.float64), 50, axis=0)
    d = rng.normal(size=o.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ib, tb, mb, _ = O.trace(ob, o, d)
    inn, tn, mn, _ = O.trace(on, o, d)
    assert np.array_equal(ib, inn) and np.array_equal(tb, tn) and np.allclose(mb, mn)
    sel = slice(0, 200)
    ip, tp = _numpy_closest(o[sel], d[sel], c2.scene.tris.astype(np.float64))
    same = ip == ib[sel]
    # a differing id is only allowed at a tie in t (coplanar overlaps) or within 1e-6 of an edge
    assert np.all(same | (np.abs(tp - tb[sel]) < 1e-9) | (mb[sel] < 1e-6))
    assert np.allclose(tp[ip >= 0], tb[sel][ip >= 0], rtol=1e-12)


def test_axis_aligned_wall_hit_distance(oracle_lib):
    os_ = O.OracleScene(Scene(tris=cube_walls(), albedo=np.full((12, 3), 0.7, np.float32), medium=Medium(0, 0, 0),
                              lights=[]), use_bvh=False)
    o = np.array([[0.25, 0.5, 0.5]])
    ids, t, _, _ = O.trace(os_, o, np.array([[-1.0, 0, 0]]))
    assert t[0] == pytest.approx(0.25, abs=1e-15) and ids[0] >= 0


# ----------------------------------------------------------------- budgets
def test_decision_budgets_are_zero_away_from_ties_and_small_overall(oracle_lib):
    c1 = W.config1()
    os_ = O.OracleScene(c1.scene)
    r = O.records(os_, c1.params, c1.positions()[:32], track_margins=1)
    L = r["L"][:, 1]
    assert np.median(r["bud_L"][:, 1] / L) < 1e-6
    assert (r["n_unc"] == 0).mean() > 0.5
    r0 = O.records(os_, c1.params, c1.positions()[:32], track_margins=0)
    for k in ("L", "grad", "hess", "radius"):
        assert np.array_equal(r[k], r0[k])                       # tracking never changes results
