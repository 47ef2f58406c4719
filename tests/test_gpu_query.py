"""GPU parity of the record grid and query kernel (Eq. radianceTaylor) against the oracle.

The query path is checked on seeded synthetic record tables (so the records are
inputs common to both sides), then end to end: GPU records -> GPU queries against
oracle records -> oracle queries.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vrc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_09258_gb300 import build
    build.build()
    import paper_1805_09258_gb300 as m
    return m


def synthetic_table(n, seed, r_lo=0.03, r_hi=0.3):
    rng = np.random.default_rng(seed)
    tab = dict(pos=rng.uniform(0.0, 1.0, size=(n, 3)), radius=rng.uniform(r_lo, r_hi, size=n),
               L=rng.uniform(0.05, 1.0, size=(n, 3)), grad=rng.normal(size=(n, 9)) * 0.5,
               hess=rng.normal(size=(n, 18)) * 2.0)
    return {k: v.astype(np.float32) for k, v in tab.items()}


def gpu_query(vrc, tab, q, order):
    recs = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in tab.items()}
    grid = vrc.Grid(recs, extrap_order=order)
    rgb, cnt = vrc.query_inscatter(grid, torch.from_numpy(np.ascontiguousarray(q)).cuda())
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), cnt.cpu().numpy(), grid


def check_query(rgb, cnt, ref, rc, near):
    ok = near == 0
    assert np.array_equal(cnt[ok], rc[ok])                      # membership is integer work: exact
    assert np.all(np.abs(cnt[~ok] - rc[~ok]) <= 2)
    hit = ok & (rc > 0)
    scale = np.abs(ref[hit]).max(axis=1, keepdims=True) + np.abs(ref[hit]) + 1e-6
    assert np.all(np.abs(rgb[hit] - ref[hit]) <= 2e-5 * scale + 1e-6)
    assert np.all(rgb[rc == 0] == 0)


@pytest.mark.parametrize("order", [1, 2])
def test_synthetic_table_parity(vrc, order):
    tab = synthetic_table(500, seed=21)
    rng = np.random.default_rng(22)
    q = np.concatenate([rng.uniform(0, 1, size=(20000, 3)), tab["pos"][:50],        # record centres
                        rng.uniform(0.98, 1.0, size=(100, 3))]).astype(np.float32)  # cube corner
    rgb, cnt, _ = gpu_query(vrc, tab, q, order)
    ref, rc, near = O.query(tab["pos"], tab["radius"], tab["L"], tab["grad"], tab["hess"], q, order=order)
    check_query(rgb, cnt, ref, rc, near)
    assert cnt.max() > 1 and (cnt == 0).any()


def test_long_cell_lists(vrc):
    """Cell lists of every length class of the grid's list sort, on a coarse grid (a block
    per cell) and on a fine one (a warp per cell: up to 64 entries in registers, up to 512 in
    a warp's shared buffer, longer lists a block each, beyond 4,096 one thread).  Records of
    radius 0.35-0.45 clustered at the centre give cells that hold thousands of records; the
    answers match the oracle and are the same bits when the grid is built twice (each list
    in record order)."""
    rng = np.random.default_rng(41)
    n = 6000
    tab = synthetic_table(n, seed=42, r_lo=0.35, r_hi=0.45)
    tab["pos"] = (0.5 + rng.normal(size=(n, 3)) * 0.08).clip(0.0, 1.0).astype(np.float32)
    # a few small records too, so that short lists exist as well
    small = synthetic_table(400, seed=43, r_lo=0.01, r_hi=0.03)
    tab = {k: np.concatenate([tab[k], small[k]]) for k in tab}
    q = rng.uniform(0.0, 1.0, size=(4000, 3)).astype(np.float32)
    for fine in (False, True):
        if fine:
            # most records small (median radius 0.02: a 64^3 grid, the warp-per-cell sort),
            # the big clustered ones still there
            tiny = synthetic_table(8000, seed=44, r_lo=0.01, r_hi=0.03)
            tab = {k: np.concatenate([tab[k], tiny[k]]) for k in tab}
        rgb, cnt, grid = gpu_query(vrc, tab, q, 1)
        rgb2, cnt2, _ = gpu_query(vrc, tab, q, 1)
        assert np.array_equal(rgb, rgb2) and np.array_equal(cnt, cnt2)
        ref, rc, near = O.query(tab["pos"], tab["radius"], tab["L"], tab["grad"], tab["hess"], q, order=1)
        check_query(rgb, cnt, ref, rc, near)
        assert cnt.max() > 4096 and (cnt < 32).any()


@pytest.mark.parametrize("order", [1, 2])
def test_exact_at_the_centre_of_a_lone_record(vrc, order):
    """Eq. radianceTaylor at a record's centre, where no other record reaches: the weight is
    w(1) = 1 and the Taylor terms vanish, so the answer is L_k itself, bit for bit (the
    oracle's pin of the same fact is in test_oracle_pins)."""
    g = (np.arange(5) + 0.5) / 5.0                     # a 5 x 5 x 5 lattice, spacing 0.2
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = pos.shape[0]
    tab = synthetic_table(n, seed=31)
    tab["pos"] = pos.astype(np.float32)
    tab["radius"] = np.random.default_rng(32).uniform(0.02, 0.099, n).astype(np.float32)   # < half the spacing
    rgb, cnt, _ = gpu_query(vrc, tab, tab["pos"], order)
    assert np.all(cnt == 1)
    assert np.array_equal(rgb, tab["L"])


def test_sizes_ragged_and_degenerate(vrc):
    rng = np.random.default_rng(23)
    for n, nq in ((1, 7), (3, 1), (33, 1000), (2049, 4097)):
        tab = synthetic_table(n, seed=n)
        q = rng.uniform(0, 1, size=(nq, 3)).astype(np.float32)
        rgb, cnt, _ = gpu_query(vrc, tab, q, 1)
        ref, rc, near = O.query(tab["pos"], tab["radius"], tab["L"], tab["grad"], None, q, order=1)
        check_query(rgb, cnt, ref, rc, near)
    # tiny radii: most queries miss; huge radii: every record covers every query
    for r_lo, r_hi in ((1e-3, 2e-3), (1.9, 2.0)):
        tab = synthetic_table(200, seed=7, r_lo=r_lo, r_hi=r_hi)
        q = rng.uniform(0, 1, size=(3000, 3)).astype(np.float32)
        rgb, cnt, _ = gpu_query(vrc, tab, q, 1)
        ref, rc, near = O.query(tab["pos"], tab["radius"], tab["L"], tab["grad"], None, q, order=1)
        check_query(rgb, cnt, ref, rc, near)


def test_zero_queries_and_empty_table(vrc):
    tab = synthetic_table(10, seed=1)
    q0 = np.zeros((0, 3), np.float32)
    rgb, cnt, grid = gpu_query(vrc, tab, q0, 1)
    assert rgb.shape == (0, 3)
    empty = {k: v[:0] for k, v in tab.items()}
    rgb, cnt, _ = gpu_query(vrc, empty, np.random.default_rng(0).uniform(0, 1, (50, 3)).astype(np.float32), 1)
    assert np.all(cnt == 0) and np.all(rgb == 0)


def test_records_then_queries_end_to_end(vrc):
    """Small workload: GPU records + GPU queries vs oracle records + oracle queries."""
    w = W.config1()
    pos = w.positions()
    q = w.queries()
    s = vrc.Scene.from_workload(w.scene)
    out = vrc.compute_records(s, torch.from_numpy(pos).cuda(), w.params)
    grid = vrc.Grid(out)
    rgb, cnt = vrc.query_inscatter(grid, torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    rgb, cnt = rgb.cpu().numpy(), cnt.cpu().numpy()
    ref = O.records(O.OracleScene(w.scene), w.params, pos, track_margins=1)
    qo, qc, near = O.query(pos, ref["radius"], ref["L"], ref["grad"], ref["hess"], q, order=1)
    # radii agree to ~1e-4, so membership may differ only for queries near a boundary
    g = to_np(out)
    rel_r = np.abs(g["radius"] - ref["radius"]) / ref["radius"]
    d = np.linalg.norm(q[:, None, :].astype(np.float64) - pos[None].astype(np.float64), axis=2)
    margin = np.abs(d - ref["radius"][None]) / ref["radius"][None]
    sensitive = (margin < 5 * rel_r.max() + 1e-5).any(axis=1)
    assert np.array_equal(cnt[~sensitive], qc[~sensitive])
    both = (~sensitive) & (qc > 0)
    assert np.all(np.abs(rgb[both] - qo[both]) <= 2e-3 * np.abs(qo[both]).max(axis=1, keepdims=True) + 1e-6)


def test_full_size_query_parity(vrc):
    """The benchmark's query call: the 4,096 records of the mid workload (the oracle's, as
    a table common to both sides) in the record grid, all 1,048,576 queries in one launch;
    131,072 of them compared element by element with the oracle's brute force."""
    w = W.config2()
    pos = w.positions()
    ref = O.records(O.OracleScene(w.scene), w.params, pos)
    tab = {"pos": pos, "radius": ref["radius"], "L": ref["L"], "grad": ref["grad"], "hess": ref["hess"]}
    tab = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in tab.items()}
    q = w.queries()
    assert q.shape[0] == 1 << 20
    rgb, cnt, _ = gpu_query(vrc, tab, q, w.params.extrap_order)
    sel = np.random.default_rng(41).choice(q.shape[0], 131072, replace=False)
    oref, rc, near = O.query(tab["pos"], tab["radius"], tab["L"], tab["grad"], tab["hess"], q[sel],
                             order=w.params.extrap_order)
    check_query(rgb[sel], cnt[sel], oref, rc, near)
    assert (rc > 0).mean() > 0.5 and rc.max() > 10


def test_rebuild_in_place_matches_a_new_grid(vrc):
    """vrc_rebuild_record_grid: one grid object rebuilt from tables of other sizes, radii and
    kinds (spheres, then ellipsoids, then spheres) answers exactly as a newly built grid."""
    rng = np.random.default_rng(61)
    q = torch.from_numpy(rng.uniform(0, 1, size=(30000, 3)).astype(np.float32)).cuda()
    grid = None
    for n, seed, r_hi, aniso in ((500, 62, 0.3, False), (3000, 63, 0.1, False), (50, 64, 0.45, True),
                                 (2000, 65, 0.2, False), (0, 66, 0.2, False)):
        tab = synthetic_table(max(n, 1), seed, r_hi=r_hi)
        tab = {k: v[:n] for k, v in tab.items()}
        if aniso:
            tab["radii"] = np.repeat(tab["radius"][:, None], 3, axis=1).astype(np.float32) * \
                np.array([1.0, 0.5, 0.8], np.float32)
            tab["axes"] = np.tile(np.eye(3, dtype=np.float32).ravel(), (n, 1))
        recs = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in tab.items()}
        fresh = vrc.Grid(recs, n=n, aniso=aniso)
        a_rgb, a_cnt = vrc.query_inscatter(fresh, q)
        if grid is None:
            grid = vrc.Grid(recs, n=n, aniso=aniso)
        else:
            grid.aniso = aniso
            grid.rebuild(recs, n=n)
        b_rgb, b_cnt = vrc.query_inscatter(grid, q)
        torch.cuda.synchronize()
        assert torch.equal(a_cnt, b_cnt) and torch.equal(a_rgb, b_rgb), (n, aniso)
