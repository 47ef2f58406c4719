"""Record parity at the headline sizes, every record (through the C ABI, GB300).

The mid workload (2,048 triangles, 4,096 records x 32 x 64 rays, the benchmark's launch)
is compared record by record with the FP64 oracle in two ways: (1) in replay mode, where
the oracle takes the GPU's discrete decisions (primary hits, FP32 ray ends, visibility)
and every record must meet the bare tolerances (radiance 1e-4 relative, gradient and
Hessian 1e-3 of their norms); (2) on the oracle's own decisions, where a record may differ
by its decision budget (the change the near-tie decisions can make, pinned by
tests/test_oracle_budget.py).  The batching workload (100,000 records of 8 x 16 ..
64 x 128 rays, 100k triangles) is compared on a block of 1,000 consecutive records of its
full launch, which spans the whole range of ray counts.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import compare_radius, compare_records, oracle_replayed, to_np

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


def test_mid_workload_every_record(vrc):
    w = W.config2()
    pos = w.positions()
    scene = vrc.Scene.from_workload(w.scene)
    d_pos = torch.from_numpy(pos).cuda()
    plain = to_np(vrc.compute_records(scene, d_pos, w.params))
    g = to_np(vrc.compute_records(scene, d_pos, w.params, debug_hits=True))
    torch.cuda.synchronize()
    for k in ("L", "grad", "hess", "radius", "status"):
        assert np.array_equal(g[k], plain[k]), k                  # the debug outputs change nothing
    osc = O.OracleScene(w.scene)
    ref = oracle_replayed(O, osc, w.params, pos, g)
    st = compare_records(g, ref)
    compare_radius(g, ref)
    assert st["n"] == 4096
    assert st["worst_L"] <= 1.0 and st["worst_g"] <= 1.0 and st["worst_H"] <= 1.0
    # the same records on the oracle's own decisions, within tolerance + decision budget
    own = O.records(osc, w.params, pos, track_margins=1)
    st2 = compare_records(g, own)
    compare_radius(g, own)
    assert st2["zero_budget"] >= 0.3 * st2["n"]


def test_batching_workload_block_of_1000(vrc):
    w = W.config3()
    pos = w.positions()
    nb = w.band_counts
    scene = vrc.Scene.from_workload(w.scene)
    full = to_np(vrc.compute_records(scene, torch.from_numpy(pos).cuda(), w.params,
                                     n_bands=torch.from_numpy(nb).cuda()))
    start, m = 41_000, 1000
    blk = slice(start, start + m)
    assert nb[blk].min() <= 10 and nb[blk].max() >= 60          # the block spans the ray-count range
    p = W.configs.replace(w.params, rec_base=start)
    g = to_np(vrc.compute_records(scene, torch.from_numpy(pos[blk].copy()).cuda(), p,
                                  n_bands=torch.from_numpy(nb[blk].copy()).cuda(), debug_hits=True))
    torch.cuda.synchronize()
    for k in ("L", "grad", "hess"):
        assert np.array_equal(g[k], full[k][blk]), k               # records do not depend on the launch
    ref = oracle_replayed(O, O.OracleScene(w.scene), w.params, pos[blk], g, rec_ids=np.arange(start, start + m),
                          n_bands=nb[blk])
    st = compare_records(full, ref, idx=np.arange(start, start + m))
    compare_radius(full, ref, idx=np.arange(start, start + m))
    assert st["n"] == m


def near_surface_positions(w, n, seed):
    """Points 1.1e-3 .. 3e-3 off the faces of the scene's boxes (outside every box): records
    whose ray sets hold sliver cells across a depth discontinuity (two vertices on the near
    face, one far away), the hardest case for the FP32 cell arithmetic."""
    rng = np.random.default_rng(seed)
    boxes = w.scene.boxes.astype(np.float64)
    out = []
    while len(out) < n:
        b = boxes[rng.integers(len(boxes))]
        ax, side = rng.integers(3), rng.integers(2)
        p = rng.uniform(b[0], b[1])
        h = rng.uniform(1.1e-3, 3e-3)
        p[ax] = b[1][ax] + h if side else b[0][ax] - h
        inside = np.all((p >= boxes[:, 0] - 1e-3) & (p <= boxes[:, 1] + 1e-3), axis=1)
        if np.all(p > 1e-3) and np.all(p < 1 - 1e-3) and not inside.any():
            out.append(p)
    return np.array(out, np.float32)


def test_records_hugging_a_surface(vrc):
    w = W.config2()
    pos = near_surface_positions(w, 256, 11)
    scene = vrc.Scene.from_workload(w.scene)
    g = to_np(vrc.compute_records(scene, torch.from_numpy(pos).cuda(), w.params, debug_hits=True))
    ref = oracle_replayed(O, O.OracleScene(w.scene), w.params, pos, g)
    st = compare_records(g, ref)
    compare_radius(g, ref)
    assert st["n"] == 256
