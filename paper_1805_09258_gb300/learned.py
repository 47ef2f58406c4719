"""Training data and training loop of the learned radius predictor (not in the paper).

Targets are the method's own output: log R of full records computed by
vrc_compute_records; inputs are the coarse features of the same positions
(vrc_coarse_features).  Training runs the library's tensor-core gradient kernel and
AdamW (vrc_mlp_train_step) over contiguous mini-batches.  Within a scene the record
positions are drawn uniformly at random; view(shuffle=True) also interleaves the scenes
(one seeded permutation of the rows), so no mini-batch comes from a single scene.  This
module only sequences library calls; examples are written into caller-sized slices.
"""
from __future__ import annotations

import numpy as np

from . import MLP, Scene, _torch, alloc_records, coarse_features, compute_records


class ExampleSet:
    """Preallocated (features [cap, 256], log radius [cap]) filled scene by scene."""

    def __init__(self, capacity: int, n_features: int = 256):
        torch = _torch()
        self.feat = torch.empty((capacity, n_features), dtype=torch.float32, device="cuda")
        self.logr = torch.empty((capacity,), dtype=torch.float32, device="cuda")
        self.n = 0
        self.cap = capacity

    def add(self, scene: Scene, positions: np.ndarray, full_params, coarse_params):
        torch = _torch()
        m = positions.shape[0]
        if self.n + m > self.cap:
            raise ValueError("example set is full")
        pos = torch.from_numpy(np.ascontiguousarray(positions, dtype=np.float32)).cuda()
        rec = alloc_records(m, full=False)
        rec["log_radius"] = self.logr[self.n:self.n + m]
        compute_records(scene, pos, full_params, out=rec)
        coarse_features(scene, pos, coarse_params, out=self.feat[self.n:self.n + m])
        self.n += m

    def view(self, shuffle: bool = False, seed: int = 0):
        if not shuffle:
            return self.feat[:self.n], self.logr[:self.n]
        torch = _torch()
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        perm = torch.randperm(self.n, generator=g, device="cuda")
        return self.feat[:self.n][perm].contiguous(), self.logr[:self.n][perm].contiguous()


def train(mlp: MLP, feat, target, steps: int, batch: int = 4096, lr: float = 2e-3, weight_decay: float = 1e-4,
          log_every: int = 0):
    """AdamW steps over contiguous mini-batches with a cosine learning-rate decay."""
    n = feat.shape[0]
    nb = max(1, n // batch)
    losses = []
    for s in range(steps):
        b = s % nb
        lo, hi = b * batch, min(n, (b + 1) * batch)
        lr_s = lr * 0.5 * (1.0 + np.cos(np.pi * s / max(1, steps)))
        want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
        loss = mlp.train_step(feat[lo:hi], target[lo:hi], lr_s, weight_decay, want_loss=want)
        if want:
            losses.append((s, loss))
    return losses
