"""Pins of the oracle's decision budgets and of its replay mode (CPU).

FP32 and FP64 may take a discrete decision of a record differently where it is a near
tie: a primary or shadow ray passing a triangle edge (Sec. 4's ray casting), a shell
vertex at its ray's end (the clamp of Sec. 4's zero-radiance samples, Sec. 6's shells).
The oracle's budget for a record is meant to be the largest change that taking such
decisions the other way can make.  Each test below builds a tiny scene where exactly one
decision is a near tie, moves the geometry across the tie, and recomputes the record in
FP64 on each side.  The change between the sides is the actual change of the flipped
decision; the budget computed on either side must cover it, and must not exceed it by more
than a factor of 4 (a budget that were, say, the whole cell's radiance would fail here).

The clamp tie is reached exactly: with the +z pole ray and a horizontal ceiling, the hit
parameter c - x_z is exact in both precisions when both lie on a 2^-28 grid, so the three
outcomes rounding can produce (vertex open at t_k; clamped below t_k; clamped at exactly
t_k, tied with the open vertices and averaged with zero radiance, reading R9) are all
realised by real geometry one float step apart.
"""
import numpy as np
import pytest

import oracle as O
from workloads.configs import RecordParams
from workloads.scenes import Medium, PointLight, Scene

MED = Medium(0.5, 0.05, 0.3)
RP = RecordParams(n_bands=8, n_bins=16)


def hess_fro(h6):
    h6 = np.asarray(h6)
    return np.sqrt(h6[..., 0] ** 2 + h6[..., 3] ** 2 + h6[..., 5] ** 2 +
                   2 * (h6[..., 1] ** 2 + h6[..., 2] ** 2 + h6[..., 4] ** 2))


def record(tris, x, light=((0.5, 0.5, 0.92), (1.0, 0.9, 0.8)), replay=None):
    tris = np.asarray(tris, np.float32)
    sc = Scene(tris=tris, albedo=np.full((tris.shape[0], 3), 0.7, np.float32), medium=MED,
               lights=[PointLight(*light)])
    return O.records(O.OracleScene(sc, use_bvh=False), RP, np.asarray([x], np.float32), track_margins=1,
                     n_threads=1, replay_hits=replay, debug=True)


def changes(a, b):
    """|a - b| per channel: radiance, gradient norm, Hessian Frobenius norm."""
    return {"L": np.abs(a["L"][0] - b["L"][0]),
            "grad": np.linalg.norm((a["grad"][0] - b["grad"][0]).reshape(3, 3), axis=1),
            "hess": hess_fro((a["hess"][0] - b["hess"][0]).reshape(3, 6))}


BUD = {"L": "bud_L", "grad": "bud_grad", "hess": "bud_hess"}


def check_budget(state, others, factor=4.0):
    """The budget of `state` covers its change to every other outcome (plus the continuous
    change of moving the geometry by a float step, < 1e-6 of the value) and is at most
    `factor` times the largest of those changes."""
    worst = {k: np.zeros(3) for k in BUD}
    for o in others:
        for k, v in changes(state, o).items():
            worst[k] = np.maximum(worst[k], v)
    for k, bk in BUD.items():
        bud = state[bk][0]
        scale = {"L": np.abs(state["L"][0]),
                 "grad": np.linalg.norm(state["grad"][0].reshape(3, 3), axis=1),
                 "hess": hess_fro(state["hess"][0].reshape(3, 6))}[k]
        assert np.all(worst[k] <= bud + 1e-6 * scale + 1e-15), (k, worst[k], bud)
        flipped = worst[k] > 1e-5 * scale
        assert np.all(bud[flipped] <= factor * worst[k][flipped]), (k, bud, worst[k])
        assert np.all(bud[~flipped] <= 1e-5 * scale[~flipped] + 1e-15), (k, bud, worst[k])
    return worst


def frame(d):
    e1 = np.cross(d, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(d, e1)


X = np.array([0.45, 0.5, 0.42])
DIRS = O.ray_directions(RP, 0)


def test_primary_ray_grazing_an_edge():
    """Ray 37 passes 3e-7 inside / outside a triangle's edge: it hits the triangle or goes on."""
    d = DIRS[37]
    p0 = X + 0.3 * d
    e1, e2 = frame(d)

    def tri(delta):
        return [[p0 + delta * e1 - 0.05 * e2, p0 + delta * e1 + 0.05 * e2, p0 + (delta - 0.08) * e1]]

    a, b = record(tri(3e-7), X), record(tri(-3e-7), X)
    assert a["hit_prim"][0, 37] == 0 and b["hit_prim"][0, 37] == -1
    assert a["n_prim_unc"][0] == 1 and b["n_prim_unc"][0] == 1
    w = check_budget(a, [b])
    check_budget(b, [a])
    assert np.all(w["L"] > 1e-4 * np.abs(a["L"][0]))          # the flip is visible in L, grad, H
    # replay: the geometry of one side with the other side's hits gives the other side's record
    ra = record(tri(3e-7), X, replay=b["hit_prim"])
    assert ra["n_replayed"][0] == 1 and ra["n_prim_unc"][0] == 0
    for k in ("L", "grad", "hess"):
        assert np.allclose(ra[k][0], b[k][0], rtol=1e-6, atol=1e-6 * np.abs(b[k][0]).max()), k
        assert np.all(ra[BUD[k]][0] == 0), k
    # replaying a record's own hits changes nothing
    rb = record(tri(-3e-7), X, replay=b["hit_prim"])
    assert rb["n_replayed"][0] == 0 and np.array_equal(rb["L"], b["L"]) and np.array_equal(rb["hess"], b["hess"])


@pytest.mark.parametrize("shell", [0, 3])
def test_shadow_ray_grazing_an_edge(shell):
    """The shadow ray of one vertex (ray 100's floor hit, or its vertex on medium shell 3)
    passes 3e-7 on either side of an occluder's edge: the vertex is lit or in shadow."""
    floor = [[[0, 0, 0.05], [1, 0, 0.05], [1, 1, 0.05]], [[0, 0, 0.05], [1, 1, 0.05], [0, 1, 0.05]]]
    d = DIRS[100]
    assert d[2] < 0
    if shell == 0:
        y = X + d * ((0.05 - X[2]) / d[2]) + np.array([0.0, 0.0, 1e-5])   # shadow rays start 1e-5 off
    else:
        y = X + d * ((shell - 0.5) * float(np.float32(0.1)))
    lp = np.array([0.5, 0.5, 0.92])
    mid = y + 0.5 * (lp - y)
    s = (lp - y) / np.linalg.norm(lp - y)
    g1, g2 = frame(s)

    def scene(delta):
        return floor + [[mid + delta * g1 - 0.03 * g2, mid + delta * g1 + 0.03 * g2, mid + (delta + 0.05) * g1]]

    a, b = record(scene(3e-7), X), record(scene(-3e-7), X)
    assert a["n_unc"][0] > 0 and b["n_unc"][0] > 0
    w = check_budget(a, [b])
    check_budget(b, [a])
    assert np.all(w["L"] > 0) and np.all(w["hess"] > 0)


def test_shell_vertex_at_its_clamp_three_outcomes():
    """The +z pole ray ends on a ceiling one float step beyond, exactly at, or one step
    short of t_1 = dt/2: open vertex, clamped vertex tied at t_1, clamped vertex below."""
    dt = float(np.float32(0.1))
    t1 = 0.5 * dt
    xz = 2.0 ** -7 + 8 * 2.0 ** -28
    c0 = xz + t1
    assert float(np.float32(xz)) == xz and float(np.float32(c0)) == c0    # exact in float32
    x = np.array([0.31, 0.27, xz])
    light = ((0.5, 0.45, 0.04), (1.0, 0.9, 0.8))

    def ceiling(c):
        return [[[0, 0, c], [1, 0, c], [0, 1, c]]]

    c = np.float32(c0)
    outs = {nm: record(ceiling(cc), x, light=light)
            for nm, cc in (("open", np.nextafter(c, np.float32(1))), ("tied", c),
                           ("below", np.nextafter(c, np.float32(0))))}
    pole = RP.n_bands * RP.n_bins
    assert outs["tied"]["hit_t"][0, pole] == t1                  # the exact tie
    assert outs["open"]["hit_t"][0, pole] > t1 > outs["below"]["hit_t"][0, pole]
    for nm, st in outs.items():
        w = check_budget(st, [o for m, o in outs.items() if m != nm])
        assert np.all(w["grad"] > 1e-3 * np.linalg.norm(st["grad"][0].reshape(3, 3), axis=1)), nm


def test_no_near_tie_no_budget():
    """A record none of whose decisions is near a tie has a zero budget."""
    floor = [[[0, 0, 0.05], [1, 0, 0.05], [1, 1, 0.05]], [[0, 0, 0.05], [1, 1, 0.05], [0, 1, 0.05]]]
    r = record(floor, X)
    assert r["n_unc"][0] == 0
    for bk in BUD.values():
        assert np.all(r[bk][0] == 0)


def test_shell_vertex_at_its_clamp_weighted_ray():
    """Ray 70 (a Monte Carlo-weighted ray) ends on a wall at t_3 (1 +- 3e-7): its vertex on
    shell 3 is open on one side and clamped on the other, which adds or removes its term of
    the Monte Carlo radiance.  The radiance budget is that term; the derivative budgets
    also cover the outcome with the clamped vertex tied at t_3, which no FP64 geometry
    reaches on a slanted ray (the pole-ray test pins it), so only the bound is checked."""
    d = DIRS[70]
    t3 = 2.5 * float(np.float32(0.1))
    f1 = np.cross(d, [0.0, 0.0, 1.0])
    f1 /= np.linalg.norm(f1)
    f2 = np.cross(d, f1)

    def wall(t_end):
        c = X + d * t_end
        return [[c - 0.3 * f1 - 0.3 * f2, c + 0.3 * f1 - 0.3 * f2, c + 0.3 * f2]]

    a, b = record(wall(t3 * (1 + 3e-7)), X), record(wall(t3 * (1 - 3e-7)), X)
    assert a["hit_t"][0, 70] > t3 > b["hit_t"][0, 70]
    for st, other in ((a, b), (b, a)):
        ch = changes(st, other)
        L = np.abs(st["L"][0])
        assert np.all(ch["L"] > 1e-5 * L)
        assert np.all(ch["L"] <= st["bud_L"][0] + 1e-6 * L)
        assert np.all(st["bud_L"][0] <= 4.0 * ch["L"])
        for k in ("grad", "hess"):
            assert np.all(ch[k] <= st[BUD[k]][0]), k


def full_replay_inputs(r):
    """A record's own decisions in the form replay mode takes them: hit ids, FP32 ray ends,
    visibility bits."""
    return dict(replay=r["hit_prim"], replay_t=r["hit_t"].astype(np.float32), replay_lit=r["lit"])


def record_replayed(tris, x, dec, light=((0.5, 0.5, 0.92), (1.0, 0.9, 0.8))):
    tris = np.asarray(tris, np.float32)
    sc = Scene(tris=tris, albedo=np.full((tris.shape[0], 3), 0.7, np.float32), medium=MED,
               lights=[PointLight(*light)])
    return O.records(O.OracleScene(sc, use_bvh=False), RP, np.asarray([x], np.float32), n_threads=1,
                     replay_hits=dec["replay"], replay_t=dec["replay_t"], replay_lit=dec["replay_lit"])


def close(a, b, rtol=1e-6):
    for k in ("L", "grad", "hess", "L_ss", "L_ms"):
        assert np.allclose(a[k], b[k], rtol=rtol, atol=rtol * np.abs(b[k]).max() + 1e-15), k


def test_full_replay_takes_the_given_visibility_and_clamp_decisions():
    """With every decision given (hits, FP32 ray ends, visibility bits) the oracle computes
    the record of the side that took them: across a shadow-ray tie, and across the three
    outcomes of the clamp tie.  Each replayed decision is a near tie here, so none is
    unexplained, and the budgets are zero."""
    floor = [[[0, 0, 0.05], [1, 0, 0.05], [1, 1, 0.05]], [[0, 0, 0.05], [1, 1, 0.05], [0, 1, 0.05]]]
    d = DIRS[100]
    y = X + d * (2.5 * float(np.float32(0.1)))
    lp = np.array([0.5, 0.5, 0.92])
    mid = y + 0.5 * (lp - y)
    s = (lp - y) / np.linalg.norm(lp - y)
    g1, g2 = frame(s)

    def scene(delta):
        return floor + [[mid + delta * g1 - 0.03 * g2, mid + delta * g1 + 0.03 * g2, mid + (delta + 0.05) * g1]]

    a, b = record(scene(3e-7), X), record(scene(-3e-7), X)
    assert not np.array_equal(a["lit"], b["lit"])
    ab = record_replayed(scene(3e-7), X, full_replay_inputs(b))
    assert ab["n_lit_replayed"][0] == 1 and ab["n_unexplained"][0] == 0
    close(ab, b)
    for bk in BUD.values():
        assert np.all(ab[bk][0] == 0)

    dt = float(np.float32(0.1))
    xz = 2.0 ** -7 + 8 * 2.0 ** -28
    c = np.float32(xz + 0.5 * dt)
    x = np.array([0.31, 0.27, xz])
    light = ((0.5, 0.45, 0.04), (1.0, 0.9, 0.8))

    def ceiling(cc):
        return [[[0, 0, cc], [1, 0, cc], [0, 1, cc]]]

    sides = {nm: record(ceiling(cc), x, light=light)
             for nm, cc in (("open", np.nextafter(c, np.float32(1))), ("tied", c),
                            ("below", np.nextafter(c, np.float32(0))))}
    for geo, cc in (("open", np.nextafter(c, np.float32(1))), ("below", np.nextafter(c, np.float32(0)))):
        for nm, st in sides.items():
            r = record_replayed(ceiling(cc), x, full_replay_inputs(st), light=light)
            assert r["n_unexplained"][0] == 0, (geo, nm)
            close(r, st, rtol=2e-6)


def test_full_replay_of_own_decisions_changes_nothing(oracle_lib):
    """Replaying a record's own decisions reproduces it (small workload, all 64 records):
    the FP32 rounding of the ray ends changes no clamp or furthest-vertex choice here."""
    import workloads as W
    w = W.config1()
    pos = w.positions()
    osc = O.OracleScene(w.scene)
    r = O.records(osc, w.params, pos, debug=True)
    rr = O.records(osc, w.params, pos, replay_hits=r["hit_prim"], replay_t=r["hit_t"].astype(np.float32),
                   replay_lit=r["lit"])
    assert np.all(rr["n_replayed"] == 0) and np.all(rr["n_lit_replayed"] == 0) and np.all(rr["n_unexplained"] == 0)
    for k in ("L", "grad", "hess", "L_ff", "radius"):
        assert np.allclose(rr[k], r[k], rtol=1e-12, atol=1e-14), k
