"""GPU parity of cache records (through the C ABI) against the FP64 oracle.

Workloads: the small one in full (64 records x 16x32 rays); the mid one at its full
size in the benchmark's launch configuration (4,096 records x 32x64 rays) with a
seeded sample of records recomputed by the oracle; ragged and chunked launches
(odd band/bin counts, several shared-memory chunks, per-record band counts); and the
edge cases (no records, an empty scene, the smallest ray sets, |A| form factors,
invalid arguments).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import compare_radius, compare_records, oracle_replayed, to_np
from workloads.configs import RecordParams

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


def run_gpu(vrc, scene, params, pos, n_bands=None, debug_hits=False, tuning=None):
    s = vrc.Scene.from_workload(scene)
    if tuning:
        s.set_tuning(**tuning)
    nbt = None if n_bands is None else torch.from_numpy(np.asarray(n_bands, np.int32)).cuda()
    out = vrc.compute_records(s, torch.from_numpy(np.ascontiguousarray(pos)).cuda(), params, n_bands=nbt,
                              debug_hits=debug_hits)
    torch.cuda.synchronize()
    return to_np(out)


def test_small_workload_all_records(vrc):
    w = W.config1()
    pos = w.positions()
    g = run_gpu(vrc, w.scene, w.params, pos)
    ref = O.records(O.OracleScene(w.scene), w.params, pos, track_margins=1)
    st = compare_records(g, ref)
    compare_radius(g, ref)
    assert st["zero_budget"] >= 0.8 * st["n"]
    assert np.allclose(g["pos"], pos)


def test_mid_workload_full_size_sampled(vrc):
    """All 4,096 records of the mid workload in one launch; 24 seeded samples re-done by the oracle."""
    w = W.config2()
    pos = w.positions()
    g = run_gpu(vrc, w.scene, w.params, pos)
    idx = np.sort(np.random.default_rng(99).choice(pos.shape[0], 24, replace=False))
    ref = O.records(O.OracleScene(w.scene), w.params, pos[idx], rec_ids=idx, track_margins=1)
    compare_records(g, ref, idx)
    compare_radius(g, ref, idx)
    assert np.all(np.isfinite(g["L"])) and np.all(np.isfinite(g["hess"]))


def test_ragged_sizes_and_chunks(vrc):
    """Odd band and bin counts, a ragged record count, and ray sets split into many chunks,
    for every block size (the default keeps the whole ray set in one chunk)."""
    w = W.config2()
    rp = RecordParams(n_bands=13, n_bins=27)
    pos = w.positions(37, seed=77)
    ref = O.records(O.OracleScene(w.scene), rp, pos, track_margins=1)
    for tuning in (None, dict(threads=128, chunk_bands=3), dict(threads=256), dict(threads=384, chunk_bands=4),
                   dict(threads=512, chunk_bands=5)):
        g = run_gpu(vrc, w.scene, rp, pos, tuning=tuning)
        compare_records(g, ref)
        compare_radius(g, ref)


def test_per_record_band_counts(vrc):
    """Uneven ray sets in one launch: record i uses n_bands[i] bands and 2 n_bands[i] bins."""
    w = W.config2()
    pos = w.positions(40, seed=78)
    nb = np.random.default_rng(5).integers(2, 14, size=40).astype(np.int32)
    rp = RecordParams(n_bands=int(nb.max()), n_bins=2 * int(nb.max()))
    g = run_gpu(vrc, w.scene, rp, pos, n_bands=nb)
    ref = O.records(O.OracleScene(w.scene), rp, pos, n_bands=nb, track_margins=1)
    compare_records(g, ref)


def test_smallest_ray_sets_and_abs_formfactor(vrc):
    w = W.config1()
    pos = w.positions(16)
    for nb, ns, signed in ((1, 3, 1), (2, 4, 1), (3, 5, 0), (8, 16, 0)):
        rp = RecordParams(n_bands=nb, n_bins=ns, ff_signed=signed)
        g = run_gpu(vrc, w.scene, rp, pos)
        ref = O.records(O.OracleScene(w.scene), rp, pos, track_margins=1)
        compare_records(g, ref)


def test_empty_scene_and_anisotropic_phase(vrc):
    """No triangles: every ray leaves the cube; strongly forward-scattering medium."""
    from workloads.scenes import Medium, PointLight, Scene
    sc = Scene(tris=np.zeros((0, 3, 3), np.float32), albedo=np.zeros((0, 3), np.float32),
               medium=Medium(0.6, 0.1, 0.8), lights=[PointLight((0.3, 0.6, 0.7), (2.0, 1.0, 0.5))])
    rp = RecordParams(n_bands=16, n_bins=32, omega_o=(0.6, 0.0, 0.8))
    pos = np.random.default_rng(3).uniform(0.05, 0.95, size=(20, 3)).astype(np.float32)
    g = run_gpu(vrc, sc, rp, pos)
    ref = O.records(O.OracleScene(sc), rp, pos, track_margins=1)
    compare_records(g, ref)
    assert np.all(g["L_ss"] == 0)


def test_zero_records_and_invalid_arguments(vrc):
    w = W.config1()
    s = vrc.Scene.from_workload(w.scene)
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    out = vrc.compute_records(s, empty, w.params)
    assert out["L"].shape == (0, 3)
    bad = RecordParams(n_bands=300, n_bins=32)
    with pytest.raises(vrc.VrcError, match="unsupported"):
        vrc.compute_records(s, torch.zeros((2, 3), dtype=torch.float32, device="cuda"), bad)
    with pytest.raises(vrc.VrcError, match="invalid"):
        vrc.compute_records(s, torch.zeros((2, 3), dtype=torch.float32, device="cuda"),
                            RecordParams(n_bands=4, n_bins=2))


def test_host_buffer_entry_point_matches_device_entry_point(vrc):
    w = W.config1()
    pos = w.positions(32)
    s = vrc.Scene.from_workload(w.scene)
    d = to_np(vrc.compute_records(s, torch.from_numpy(pos).cuda(), w.params))
    h = vrc.compute_records_host(s, pos, w.params)
    for k in ("L", "grad", "hess", "radius", "status"):
        assert np.array_equal(h[k], d[k]), k


def test_whole_step_from_host_buffers_matches_device_calls(vrc):
    """vrc_cache_step_host (host positions and points in; records and query answers out,
    copies inside the call) gives, bit for bit, what the device calls give: records as
    vrc_compute_records, answers as vrc_build_record_grid + vrc_query_inscatter; also on a
    second call, which rebuilds the grid in place."""
    w = W.config2()
    step = vrc.HostStep(vrc.Scene.from_workload(w.scene), w.params)
    s = vrc.Scene.from_workload(w.scene)
    for seed in (5, 6):
        pos = w.positions(500, seed=seed)
        q = w.queries(40000, seed=seed)
        out = {"L": np.zeros((500, 3), np.float32), "grad": np.zeros((500, 9), np.float32),
               "hess": np.zeros((500, 18), np.float32), "radius": np.zeros(500, np.float32),
               "status": np.zeros(500, np.int32), "rgb": np.zeros((40000, 3), np.float32),
               "qstatus": np.zeros(40000, np.int32)}
        step(pos, q, out)
        d = vrc.compute_records(s, torch.from_numpy(pos).cuda(), w.params)
        rgb, cnt = vrc.query_inscatter(vrc.Grid(d, extrap_order=w.params.extrap_order), torch.from_numpy(q).cuda())
        torch.cuda.synchronize()
        d = to_np(d)
        for k in ("L", "grad", "hess", "radius", "status"):
            assert np.array_equal(out[k], d[k]), (seed, k)
        assert np.array_equal(out["rgb"], rgb.cpu().numpy()) and np.array_equal(out["qstatus"], cnt.cpu().numpy())
        assert (out["qstatus"] > 0).mean() > 0.5


def test_hit_ids_agree_except_near_edges(vrc):
    """Primary hit primitive ids agree on >= 99.99% of rays; a mismatch is allowed only
    where the oracle's ray passes within 1e-5 of a triangle edge (or meets two
    coplanar triangles at the same t)."""
    total = mism = 0
    for w, n in ((W.config1(), 64), (W.config2(), 16)):
        pos = w.positions(n)
        g = run_gpu(vrc, w.scene, w.params, pos, debug_hits=True)
        ref = O.records(O.OracleScene(w.scene), w.params, pos, track_margins=1, debug=True)
        V = w.params.n_rays
        gh, oh = g["hit_prim"][:, :V], ref["hit_prim"][:, :V]
        bad = gh != oh
        total += gh.size
        mism += int(bad.sum())
        ok_tie = (ref["hit_margin"][:, :V] < 1e-5) | (ref["hit_tie"][:, :V] < 1e-5)
        assert np.all(ok_tie[bad]), np.argwhere(bad & ~ok_tie)[:5]
        same = ~bad
        assert np.allclose(g["hit_t"][:, :V][same], ref["hit_t"][:, :V][same], rtol=2e-5, atol=1e-6)
    assert mism <= 1e-4 * total + 1


def test_light_buffer_shadow_rays_match_bvh_shadow_rays(vrc):
    """Shadow rays through the light buffer test the same triangles with the same predicate
    as BVH any-hit traversal, and its per-cell shortcuts (nearer than every candidate: lit;
    behind a triangle covering the cell: shadowed) give the same answers: records must agree
    (to float summation order), also on the tessellated 250k-triangle scene."""
    for w, n in ((W.config1(), 64), (W.config2(), 256), (W.config5(), 64)):
        pos = w.positions(n)
        a = run_gpu(vrc, w.scene, w.params, pos, tuning=dict(shadow_bvh=0))
        b = run_gpu(vrc, w.scene, w.params, pos, tuning=dict(shadow_bvh=1))
        same = np.all(a["L"] == b["L"], axis=1)
        assert same.mean() > 0.95
        for k in ("L", "grad", "hess"):
            diff = np.abs(a[k] - b[k]).max(axis=1)
            scale = np.abs(b[k]).max(axis=1) + 1e-12
            assert np.mean(diff <= 1e-5 * scale) > 0.95, k


def test_single_and_multiple_scattering_parts(vrc):
    """parts = 1 (surface shell) and parts = 2 (medium shells) give the single- and
    multiple-scattering records of Sec. 6's two caches: bit for bit the parts of the whole
    record, and their radii follow their own luminance and Hessian (oracle, Eq.
    radiusAniso3D)."""
    w = W.config1()
    pos = w.positions()
    whole = run_gpu(vrc, w.scene, w.params, pos)
    ref = O.records(O.OracleScene(w.scene), w.params, pos, track_margins=1)
    Y = np.array([0.2126, 0.7152, 0.0722])
    for parts, sfx in ((1, "_ss"), (2, "_ms")):
        p = W.configs.replace(w.params, parts=parts)
        g = run_gpu(vrc, w.scene, p, pos)
        for k in ("L", "grad", "hess"):
            assert np.array_equal(g[k], whole[k + sfx]), (parts, k)
            assert np.array_equal(g[k + sfx], whole[k + sfx]), (parts, k)
        other = "_ms" if parts == 1 else "_ss"
        assert np.all(g["L" + other] == 0) and np.all(g["hess" + other] == 0)
        if parts == 1:
            assert np.all(g["n_shells"] == 0)
        # radius of the part from the oracle's part (tolerances as for the whole record)
        part_ref = dict(ref)
        part_ref["L"], part_ref["hess"] = ref["L" + sfx], ref["hess" + sfx]
        for r in range(pos.shape[0]):
            LY = float(Y @ ref["L" + sfx][r])
            hy = (Y[:, None] * ref["hess" + sfx][r].reshape(3, 6)).sum(0)
            R, st, lam = O.radius(LY, hy, p.eps, p.r_min, p.r_max)
            part_ref.setdefault("_R", []).append(R)
            part_ref.setdefault("_lam", []).append(np.abs(lam).max())
            part_ref.setdefault("_LY", []).append(LY)
            part_ref.setdefault("_st", []).append(st)
        part_ref["radius"] = np.array(part_ref["_R"])
        part_ref["lam_max"] = np.array(part_ref["_lam"])
        part_ref["L_Y"] = np.array(part_ref["_LY"])
        part_ref["status"] = np.array(part_ref["_st"])
        compare_radius(g, part_ref)
    invalid = W.configs.replace(w.params, parts=3)
    with pytest.raises(vrc.VrcError):
        run_gpu(vrc, w.scene, invalid, pos[:2])


def test_out_of_range_band_counts_are_flagged_not_computed(vrc):
    """A per-record band count outside [2, params n_bands] would overrun the shared buffers
    sized for params n_bands: such records are skipped with status VRC_REC_BAD_COUNT while
    the others are computed as usual."""
    w = W.config1()
    pos = w.positions(6, seed=17)
    p = RecordParams(n_bands=8, n_bins=16)
    nb = np.array([4, 9, 1, 8, 0, 6], np.int32)          # 9 > 8, 1 < 2, 0 < 2: bad
    g = run_gpu(vrc, w.scene, p, pos, n_bands=nb)
    bad = np.array([False, True, True, False, True, False])
    assert np.all((g["status"][bad] & 16) != 0) and np.all((g["status"][~bad] & 16) == 0)
    assert np.all(g["L"][bad] == 0) and np.all(g["hess"][bad] == 0)
    good = np.flatnonzero(~bad)
    for i in good:
        one = run_gpu(vrc, w.scene, W.configs.replace(p, n_bands=int(nb[i]), n_bins=2 * int(nb[i]), rec_base=int(i)),
                      pos[i:i + 1])
        assert np.array_equal(g["L"][i], one["L"][0]) and np.array_equal(g["hess"][i], one["hess"][0])


def test_prepass_matches_in_kernel_tracing(vrc):
    """The primary-ray pre-pass (a flat kernel that traces ahead of the record kernel) gives
    the records the record kernel computes when it traces its own primary rays."""
    w = W.config2()
    pos = w.positions(300, seed=23)
    a = run_gpu(vrc, w.scene, w.params, pos)
    b = run_gpu(vrc, w.scene, w.params, pos, tuning=dict(no_prepass=1))
    for k in ("L", "grad", "hess", "radius"):
        x, y = a[k].astype(np.float64), b[k].astype(np.float64)
        assert np.max(np.abs(x - y)) <= 1e-6 * np.abs(y).max() + 1e-12, k
    assert np.array_equal(a["n_cells"], b["n_cells"])
    # debug hit ids are written by the pre-pass in the same layout
    a = run_gpu(vrc, w.scene, w.params, pos[:8], debug_hits=True)
    b = run_gpu(vrc, w.scene, w.params, pos[:8], debug_hits=True, tuning=dict(no_prepass=1))
    assert np.array_equal(a["hit_prim"], b["hit_prim"]) and np.array_equal(a["hit_t"], b["hit_t"])


def test_prepass_in_batches_matches_in_kernel_tracing(vrc):
    """33,000 records of 2,050 rays exceed the pre-pass buffers (64 Mi rays), so the launch
    runs as two batches of work items; the records equal those the record kernel computes
    when it traces its own primary rays."""
    w = W.config2()
    pos = w.positions(33000, seed=29)
    a = run_gpu(vrc, w.scene, w.params, pos)
    b = run_gpu(vrc, w.scene, w.params, pos, tuning=dict(no_prepass=1))
    for k in ("L", "grad", "hess", "radius", "status", "n_cells"):
        assert np.array_equal(a[k], b[k]), k


def test_largest_ray_set(vrc):
    """The largest ray set the record kernel takes, 256 bands x 512 bins (131,074 rays, in
    band chunks), on the small scene: three records against the oracle replaying the GPU's
    decisions, at the bare tolerances; one more band is refused."""
    w = W.config1()
    rp = RecordParams(n_bands=256, n_bins=512)
    pos = w.positions(3, seed=23)
    g = run_gpu(vrc, w.scene, rp, pos, debug_hits=True)
    ref = oracle_replayed(O, O.OracleScene(w.scene), rp, pos, g)
    st = compare_records(g, ref)
    compare_radius(g, ref)
    assert st["n"] == 3 and st["worst_L"] <= 1.0 and st["worst_g"] <= 1.0 and st["worst_H"] <= 1.0
    with pytest.raises(vrc.VrcError, match="unsupported"):
        run_gpu(vrc, w.scene, RecordParams(n_bands=257, n_bins=512), pos)


def test_many_small_ray_sets_in_128_thread_blocks(vrc):
    """1,000 records of 16 x 32 rays (enough to fill six 128-thread blocks per SM, the
    launch shape such sets get by default) on the small scene: a sample of 64 against the
    oracle replaying the GPU's decisions, at the bare tolerances, and every record equal to
    the 384-thread launch up to the order of the sums."""
    w = W.config1()
    pos = w.positions(1000, seed=29)
    g = run_gpu(vrc, w.scene, w.params, pos, debug_hits=True)
    sel = np.arange(3, 1000, 16)
    ref = oracle_replayed(O, O.OracleScene(w.scene), w.params, pos[sel], g, rec_ids=sel, idx=sel)
    st = compare_records(g, ref, idx=sel)
    assert st["worst_L"] <= 1.0 and st["worst_g"] <= 1.0 and st["worst_H"] <= 1.0
    g384 = run_gpu(vrc, w.scene, w.params, pos, tuning=dict(threads=384))
    for k in ("L", "grad", "hess"):
        scale = np.abs(g384[k]).max(axis=1, keepdims=True) + 1e-30
        assert np.all(np.abs(g[k] - g384[k]) <= 1e-4 * scale), k
