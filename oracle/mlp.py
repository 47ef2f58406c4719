"""FP64 oracle of the learned radius predictor (not in the paper; test infrastructure only).

Network: x (256) -> z1 = W1 x + b1 (64) -> h1 = gelu(z1) -> z2 = W2 h1 + b2 (64) ->
h2 = gelu(z2) -> y = w3 . h2 + b3, the predicted log radius; loss = mean (y - t)^2
over the batch.  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.

`quantize=True` models the tensor-core kernels' BF16 operand rounding points, so the
oracle and the GPU round the same quantities: the input x, W1, W2 and w3 are BF16;
h1 is rounded to BF16 before the second layer; in the backward pass dz2 is rounded
to BF16 where it is a GEMM operand (dh1 = dz2 W2 and dW2 = dz2^T h1) and dz1 where it
is one (dW1 = dz1^T x).  Everything else is FP64.  `quantize=False` is the plain
network, used for the finite-difference pins.

Parameter vector layout (shared with the C ABI): W1 [64][256], b1 [64], W2 [64][64],
b2 [64], w3 [64], b3 [1]: 20,673 floats.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

D_IN, D_H = 256, 64
SIZES = [("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)), ("w3", (D_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SIZES])


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters (He-style normal weights, zero biases), float32-exact."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, math.sqrt(2.0 / D_IN), (D_H, D_IN)), "b1": np.zeros(D_H),
         "W2": rng.normal(0, math.sqrt(2.0 / D_H), (D_H, D_H)), "b2": np.zeros(D_H),
         "w3": rng.normal(0, math.sqrt(1.0 / D_H), D_H), "b3": np.full(1, -1.5)}
    return pack(p).astype(np.float32).astype(np.float64)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, x, quantize=True):
    """Returns y [n] and the intermediates of the forward pass."""
    p = unpack(theta)
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    X = q(x)
    W1, W2, w3 = q(p["W1"]), q(p["W2"]), q(p["w3"])
    z1 = X @ W1.T + p["b1"]
    h1 = gelu(z1)
    h1q = q(h1)
    z2 = h1q @ W2.T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ w3 + p["b3"][0]
    return y, dict(X=X, W1=W1, W2=W2, w3=w3, z1=z1, h1q=h1q, z2=z2, h2=h2)


def loss_and_grad(theta, x, t, quantize=True):
    """MSE loss over the batch and its gradient with respect to the parameter vector."""
    n = x.shape[0]
    y, c = forward(theta, x, quantize)
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    dz2 = (dy[:, None] * c["w3"][None, :]) * gelu_prime(c["z2"])
    dz2q = q(dz2)
    dh1 = dz2q @ c["W2"]
    dz1 = dh1 * gelu_prime(c["z1"])
    dz1q = q(dz1)
    g = {"W1": dz1q.T @ c["X"], "b1": dz1.sum(0), "W2": dz2q.T @ c["h1q"], "b2": dz2.sum(0),
         "w3": c["h2"].T @ dy, "b3": np.array([dy.sum()])}
    return loss, pack(g)


def adamw(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov & Hutter): decoupled weight decay on every parameter."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
