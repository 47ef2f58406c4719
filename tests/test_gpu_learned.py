"""The learned radius predictor end to end: trained on GPU on records the method itself
computes (mid-style scenes), it predicts held-out radii, and learned placement covers the
same candidates with fewer full records than plain placement at the same error."""
import numpy as np
import pytest

import oracle.mlp as M
import workloads as W
from workloads.configs import RecordParams

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

COARSE = RecordParams(n_bands=8, n_bins=16, seed=1003)


@pytest.fixture(scope="module")
def vrc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_09258_gb300 import build
    build.build()
    import paper_1805_09258_gb300 as m
    return m


@pytest.fixture(scope="module")
def trained(vrc):
    from paper_1805_09258_gb300 import learned
    ex = learned.ExampleSet(8 * 8192)
    for seed in range(1, 9):
        w = W.config4(scene_seed=seed)
        ex.add(vrc.Scene.from_workload(w.scene), w.positions(8192, seed=100 + seed), w.params, COARSE)
    F, T = ex.view()
    mlp = vrc.MLP(M.init_params(21))
    losses = learned.train(mlp, F, T, steps=1500, batch=4096, lr=2e-3, log_every=500)
    return mlp, losses


def test_predicts_held_out_radii(vrc, trained):
    from paper_1805_09258_gb300 import learned
    mlp, losses = trained
    w = W.config4(scene_seed=40)
    ex = learned.ExampleSet(8192)
    ex.add(vrc.Scene.from_workload(w.scene), w.positions(8192, seed=400), w.params, COARSE)
    f, t = ex.view()
    pred = mlp.predict(f).cpu().numpy().astype(np.float64)
    t = t.cpu().numpy().astype(np.float64)
    mse = float(np.mean((pred - t) ** 2))
    r2 = 1.0 - mse / float(np.var(t))
    print("held-out log-radius mse", mse, "r2", r2, "losses", losses)
    assert losses[-1][1] < losses[0][1]
    assert r2 > 0.3, (mse, r2)
    assert mlp.status() == 0


def test_learned_placement_needs_fewer_records_at_equal_error(vrc, trained):
    """Coverage is decided by the full records' true radii in both cases, so both placements
    honour the error tolerance; the predictor's levels alone (no coarse-record fallback) put
    the coarse-wave sites where the predicted radius is large (cell up to 1.5 x radius) and
    need fewer records."""
    from paper_1805_09258_gb300 import placement
    mlp = trained[0]
    w = W.config4(scene_seed=41)
    s = vrc.Scene.from_workload(w.scene)
    cand = torch.from_numpy(w.positions(60000, seed=441)).cuda()
    plain = placement.place(s, w.params, cand)
    learn = placement.place(s, w.params, cand, mlp=mlp, coarse_params=COARSE, cell_over_radius=1.5, fallback=False)
    for r in (plain, learn):
        _, cnt = vrc.query_inscatter(r.grid, cand)
        assert int((cnt == 0).sum()) == 0
    print("records plain", plain.n_records, plain.waves, "learned", learn.n_records, learn.waves)
    assert learn.n_records < 0.9 * plain.n_records, (learn.n_records, plain.n_records)
    # equal error: interpolation error against full records at a sample of candidates
    idx = torch.arange(0, cand.shape[0], 97, device="cuda")
    q = cand[idx].contiguous()
    ref = vrc.compute_records(s, q, w.params, full=False)["L"].cpu().numpy()
    errs = []
    for r in (plain, learn):
        rgb, _ = vrc.query_inscatter(r.grid, q)
        e = np.linalg.norm(rgb.cpu().numpy() - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-6)
        errs.append(float(np.median(e)))
    print("median relative interpolation error plain / learned", errs)
    assert errs[1] <= 1.5 * errs[0] + 0.02, errs


def test_fallback_rule_and_one_shot_placement(vrc, trained):
    """The coarse-record check (the error at the predicted radius by the coarse ray set's
    own Hessian, Eq. radiusAniso3D, within the tolerance) keeps exactly the predictions
    not larger than the coarse record's radius: the placement's fallback count equals the
    count computed here from the same predictions and coarse records.  Learned placement
    with the fallback, one-shot or by waves, still covers every candidate, and at a
    tolerance of eps / 10 the predictions are carried there by (1/5) log 0.1."""
    import dataclasses
    from paper_1805_09258_gb300 import placement
    mlp = trained[0]
    w = W.config4(scene_seed=41)
    s = vrc.Scene.from_workload(w.scene)
    cand = torch.from_numpy(w.positions(60000, seed=441)).cuda()
    for eps in (w.params.eps, w.params.eps / 10):
        rp = W.configs.replace(w.params, eps=eps)
        for one_shot in (False, True):
            r = placement.place(s, rp, cand, mlp=mlp, coarse_params=COARSE, cell_over_radius=1.5,
                                eps_train=w.params.eps, one_shot=one_shot)
            _, cnt = vrc.query_inscatter(r.grid, cand)
            assert int((cnt == 0).sum()) == 0
            assert r.predicted_sites > 1000
        # the rule, independently: the same prediction sites (one per cell of the 2^5 grid)
        level = torch.full((cand.shape[0],), 2, dtype=torch.int32, device="cuda")
        scratch = torch.empty((8 ** 8 + 2 * cand.shape[0] + cand.shape[0] // 1024 + 2,), dtype=torch.int32,
                              device="cuda")
        site_idx = torch.empty((cand.shape[0],), dtype=torch.int32, device="cuda")
        site_pts = torch.empty((cand.shape[0], 3), dtype=torch.float32, device="cuda")
        m = vrc.select_sites(cand, level, 5, scratch, site_idx, site_pts)
        # the pool size it reports: every candidate, then those left after retiring a third
        m2, pool = vrc.select_sites(cand, level, 5, scratch, site_idx, site_pts, with_pool=True)
        assert m2 == m and pool == cand.shape[0]
        lv2 = level.clone()
        lv2[::3] = -1
        _, pool2 = vrc.select_sites(cand, lv2, 5, scratch, site_idx, site_pts, with_pool=True)
        assert pool2 == int((lv2 >= 0).sum())
        m = vrc.select_sites(cand, level, 5, scratch, site_idx, site_pts)     # the sites again
        pts = site_pts[:m].contiguous()
        pred = mlp.predict(vrc.coarse_features(s, pts, COARSE)).cpu().numpy().astype(np.float64)
        pred += 0.2 * np.log(eps / w.params.eps)
        cp = dataclasses.replace(rp, n_bands=COARSE.n_bands, n_bins=COARSE.n_bins, seed=COARSE.seed)
        rc = vrc.compute_records(s, pts, cp, full=False)["radius"].cpu().numpy().astype(np.float64)
        want = int(np.sum(~(np.exp(pred) <= rc * (1 + 1e-6))))
        assert m == r.predicted_sites
        assert abs(r.fallback_sites - want) <= max(2, m // 1000), (r.fallback_sites, want, m)


def test_multi_level_sites_and_batched_placement(vrc, trained):
    """One selection pass over several levels picks, in every (level, cell) of the candidates'
    own levels, the smallest candidate index (checked against numpy); the pool count and
    the level bump do what they say; batched learned placement (each wave over all levels,
    uncovered candidates one level finer after it) covers every candidate."""
    from paper_1805_09258_gb300 import placement
    rng = np.random.default_rng(9)
    n = 5000
    pts_np = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    lev_np = rng.integers(0, 9, size=n).astype(np.int32) - 1            # -1 .. 7
    lev_np[lev_np == 0] = -1
    lev_np[lev_np == 1] = 2
    pts = torch.from_numpy(pts_np).cuda()
    level = torch.from_numpy(lev_np).cuda()
    scratch = torch.empty(((8 ** 8 - 8 ** 2) // 7 + 2 * n + n // 1024 + 3,), dtype=torch.int32, device="cuda")
    site_idx = torch.empty((n,), dtype=torch.int32, device="cuda")
    site_pts = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    m, pool = vrc.select_sites_levels(pts, level, 2, 7, scratch, site_idx, site_pts)
    best = {}
    for i in range(n):
        l = int(lev_np[i])
        if 2 <= l <= 7:
            g = 1 << l
            c = tuple(np.minimum(np.floor(pts_np[i] * np.float32(g)).astype(np.int64), g - 1))
            best.setdefault((l, c), i)
    want = sorted(best.values())
    got = site_idx[:m].cpu().numpy()
    assert m == len(want) and np.array_equal(got, want)
    assert np.array_equal(site_pts[:m].cpu().numpy(), pts_np[want])
    assert pool == int((lev_np >= 0).sum())
    vrc.bump_levels(level, 8)
    assert np.array_equal(level.cpu().numpy(), np.where(lev_np >= 0, np.minimum(lev_np + 1, 8), -1))

    mlp = trained[0]
    w = W.config4(scene_seed=41)
    s = vrc.Scene.from_workload(w.scene)
    cand = torch.from_numpy(w.positions(60000, seed=441)).cuda()
    for eps in (w.params.eps, w.params.eps / 10):
        rp = W.configs.replace(w.params, eps=eps)
        r = placement.place(s, rp, cand, mlp=mlp, coarse_params=COARSE, cell_over_radius=1.5,
                            eps_train=w.params.eps, predict_level=3, batched=True)
        _, cnt = vrc.query_inscatter(r.grid, cand)
        assert int((cnt == 0).sum()) == 0
        assert any(wv[0] == "levels" for wv in r.waves)
