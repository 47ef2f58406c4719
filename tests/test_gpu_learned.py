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
    """Coverage is judged by the full records' true radii in both cases, so both placements
    honour the error tolerance; the learned one puts the coarse-wave sites where the
    predicted radius is large (cell up to 1.5 x radius) and needs fewer records."""
    from paper_1805_09258_gb300 import placement
    mlp = trained[0]
    w = W.config4(scene_seed=41)
    s = vrc.Scene.from_workload(w.scene)
    cand = torch.from_numpy(w.positions(60000, seed=441)).cuda()
    plain = placement.place(s, w.params, cand)
    learn = placement.place(s, w.params, cand, mlp=mlp, coarse_params=COARSE, cell_over_radius=1.5)
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
