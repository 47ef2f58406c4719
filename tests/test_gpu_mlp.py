"""GPU parity of the learned radius predictor: coarse features, the tensor-core MLP's
forward pass and gradients against the FP64 oracle (which rounds the same operands to
BF16), training progress, and bit-exact checkpoint/resume."""
import numpy as np
import pytest

import oracle as O
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


def realistic_features(n, seed):
    rng = np.random.default_rng(seed)
    f = np.concatenate([rng.normal(-1.2, 0.6, (n, 128)), rng.uniform(0, 1, (n, 128))], axis=1)
    return f.astype(np.float32)


def perturbed_params(seed):
    rng = np.random.default_rng(seed)
    th = M.init_params(seed)
    return (th + rng.normal(0, 0.05, th.shape)).astype(np.float32)


def test_coarse_features_match_oracle(vrc):
    w = W.config2()
    pos = w.positions(48, seed=31)
    s = vrc.Scene.from_workload(w.scene)
    g = vrc.coarse_features(s, torch.from_numpy(pos).cuda(), COARSE).cpu().numpy().astype(np.float64)
    ref, unc = O.coarse_features(O.OracleScene(w.scene), COARSE, pos)
    N = 128
    ok_log = np.abs(g[:, :N] - ref[:, :N]) <= 2e-5
    ok_tv = np.abs(g[:, N:] - ref[:, N:]) <= 2e-5 * np.maximum(np.abs(ref[:, N:]), 1e-2)
    ok = np.concatenate([ok_log, ok_tv], axis=1)
    assert np.all(ok | unc), np.argwhere(~(ok | unc))[:5]
    assert unc.mean() < 0.01


def test_mlp_forward_matches_oracle(vrc):
    theta = perturbed_params(3)
    x = realistic_features(300, 4)                       # three tiles, the last one ragged
    mlp = vrc.MLP(theta)
    y = mlp.predict(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    yr, _ = M.forward(theta.astype(np.float64), x, quantize=True)
    err = np.abs(y - yr)
    # same BF16 rounding points on both sides; differences come from FP32 accumulation
    # and the rare h1 element that rounds to the other neighbouring BF16 value
    assert np.max(err) <= 5e-3 * (1.0 + np.abs(yr).max()), np.max(err)
    assert np.median(err) <= 2e-4 * (1.0 + np.abs(yr).max())
    assert mlp.status() == 0


def test_mlp_gradient_matches_oracle_and_is_deterministic(vrc):
    theta = perturbed_params(5)
    x = realistic_features(300, 6)
    t = np.random.default_rng(7).normal(-1.6, 0.4, 300).astype(np.float32)
    mlp = vrc.MLP(theta)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    g1, pred = mlp.gradient(X, T)
    g2, _ = mlp.gradient(X, T)
    g1, g2 = g1.cpu().numpy().astype(np.float64), g2.cpu().numpy()
    assert np.array_equal(g1.astype(np.float32), g2)                        # bitwise reproducible
    loss, gr = M.loss_and_grad(theta.astype(np.float64), x, t, quantize=True)
    o = 0
    for name, shp in M.SIZES:
        k = int(np.prod(shp))
        a, b = g1[o:o + k], gr[o:o + k]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-7, (name, np.linalg.norm(a - b),
                                                                          np.linalg.norm(b))
        o += k
    yr, _ = M.forward(theta.astype(np.float64), x, quantize=True)
    assert np.max(np.abs(pred.cpu().numpy() - yr)) <= 5e-3 * (1.0 + np.abs(yr).max())


def test_training_reduces_loss_and_resumes_bit_exactly(vrc):
    teacher = perturbed_params(11).astype(np.float64)
    x = realistic_features(2048, 12)
    t, _ = M.forward(teacher, x, quantize=False)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda()
    init = M.init_params(13).astype(np.float32)
    a = vrc.MLP(init)
    first = a.train_step(X, T, lr=3e-3, want_loss=True)
    ckpt = None
    for step in range(2, 61):
        a.train_step(X, T, lr=3e-3)
        if step == 30:
            ckpt = a.get_params(with_moments=True)
    last = a.train_step(X, T, lr=3e-3, want_loss=True)
    assert last < 0.3 * first, (first, last)
    b = vrc.MLP(init)
    b.set_params(*ckpt[:3], step=ckpt[3])
    for step in range(31, 61):
        b.train_step(X, T, lr=3e-3)
    b.train_step(X, T, lr=3e-3)
    pa, pb = a.get_params(), b.get_params()
    assert np.array_equal(pa, pb)


def test_bf16_features_and_tma_forward(vrc):
    """BF16 features (vrc_coarse_features_bf16) are the FP32 features rounded to nearest
    even, bit for bit; the forward pass that reads them by tiled TMA copies
    (vrc_mlp_predict_bf16) gives, bit for bit, the FP32 path's predictions (whose staging
    rounds the same features the same way), for ragged sizes over one and many tiles."""
    w = W.config4()
    s = vrc.Scene.from_workload(w.scene)
    pos = torch.from_numpy(w.positions(3000, seed=71)).cuda()
    f32 = vrc.coarse_features(s, pos, COARSE)
    b16 = vrc.coarse_features(s, pos, COARSE, bf16=True)
    assert b16.dtype == torch.bfloat16
    assert torch.equal(b16, f32.to(torch.bfloat16))
    mlp = vrc.MLP(perturbed_params(3))
    for n in (1, 127, 128, 129, 3000):
        a = mlp.predict(f32[:n].contiguous())
        b = mlp.predict(b16[:n].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(a, b), n
    big = torch.from_numpy(realistic_features(70001, 9)).cuda()
    a = mlp.predict(big)
    b = mlp.predict(big.to(torch.bfloat16).contiguous())
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert mlp.status() == 0
