"""Pins of the learned-radius oracle (the MLP and its coarse features are not in the paper).

P10: the FP64 gradient of the MSE loss against central finite differences; the BF16
rounding helper against the bit-level definition; AdamW against its closed form on a
quadratic; the coarse features against direct geometry."""
import math

import numpy as np

import oracle as O
import oracle.mlp as M
import workloads as W
from workloads.configs import RecordParams


def test_bf16_rounding_matches_the_bit_definition():
    x = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -3.14159, 1e-30, 65504.0, 0.0])
    r = M.bf16(x)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert r[0] == 1.0 and r[1] == 1.0 and r[3] == 1.0078125
    assert abs(r[4] - (-3.140625)) < 1e-12
    assert r[7] == 0.0
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_mlp_gradient_vs_finite_differences():
    rng = np.random.default_rng(0)
    theta = M.init_params(1)
    x = rng.normal(size=(16, M.D_IN)) * 0.5
    t = rng.normal(size=16) * 0.3 - 1.5
    loss, g = M.loss_and_grad(theta, x, t, quantize=False)
    idx = np.concatenate([rng.choice(M.D_H * M.D_IN, 40, replace=False),
                          np.arange(M.D_H * M.D_IN, M.N_PARAMS)[::97], [M.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, x, t, quantize=False)[0] - M.loss_and_grad(theta - e, x, t, quantize=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_gelu_derivative_and_values():
    z = np.linspace(-5, 5, 101)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(M.gelu_prime(z), fd, atol=1e-8)
    assert abs(M.gelu(1.0) - 0.8413447460685429) < 1e-15          # 1 * Phi(1)


def test_adamw_first_step_moves_each_parameter_by_lr():
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -0.1, 2.0])
    th, m, v = M.adamw(theta, np.zeros(3), np.zeros(3), g, 1, lr=0.01, wd=0.0)
    # with bias correction the first step is lr * g / |g| (eps negligible)
    assert np.allclose(th, theta - 0.01 * np.sign(g), atol=1e-9)


def test_coarse_features_against_direct_geometry():
    """Empty room: log distance to the wall; transmittance to the light (no occluders)."""
    from workloads.scenes import Medium, PointLight, Scene, cube_walls
    sc = Scene(tris=cube_walls(), albedo=np.full((12, 3), 0.7, np.float32), medium=Medium(0.5, 0.3, 0.0),
               lights=[PointLight((0.5, 0.5, 0.92), (1, 1, 1))])
    rp = RecordParams(n_bands=8, n_bins=16, seed=1003)
    pos = np.array([[0.3, 0.4, 0.5]], np.float32)
    f, unc = O.coarse_features(O.OracleScene(sc), rp, pos)
    d = O.ray_directions(rp, rec=0)[:128]
    x = pos[0].astype(np.float64)
    with np.errstate(divide="ignore"):
        tp = np.where(d > 0, (1 - x) / d, np.where(d < 0, -x / d, np.inf))
    te = tp.min(axis=1)
    assert np.allclose(f[0, :128], np.log(te), atol=1e-12)
    y = x + te[:, None] * d
    lp = np.array([0.5, 0.5, 0.92], np.float32).astype(np.float64)
    st = float(np.float32(0.5)) + float(np.float32(0.3))
    assert np.allclose(f[0, 128:], np.exp(-st * np.linalg.norm(lp - y, axis=1)), rtol=1e-9)
