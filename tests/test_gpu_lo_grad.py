"""Parity of the lo_grad record option (GB300, through the C ABI): a medium vertex's outgoing
radiance varies with x through the HG phase of the light it scatters toward x, so the
record's gradient and Hessian keep grad L_o and H L_o (Eq. reducedRadianceDerivatives
without Sec. 4's constant-L_o simplification; Sec. 7 discusses it).

Checked against the FP64 oracle with the same option in replay mode (the GPU's discrete
decisions, bare tolerances), on the small workload (every record) and on a sample of the
mid workload's full launch; the radiance itself is the same bits as without the option
(the factor is 1 at the record centre), single scattering is unchanged to rounding, and a
scene with more than one light is refused."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import compare_records, oracle_replayed, to_np
from workloads.configs import replace
from workloads.scenes import PointLight

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


def _run(vrc, w, rp, pos, debug_hits=False):
    s = vrc.Scene.from_workload(w.scene)
    out = vrc.compute_records(s, torch.from_numpy(np.ascontiguousarray(pos)).cuda(), rp, debug_hits=debug_hits)
    torch.cuda.synchronize()
    return to_np(out)


def _check(vrc, w, idx=None):
    pos = w.positions()
    rp = replace(w.params, lo_grad=1)
    g = _run(vrc, w, rp, pos, debug_hits=True)
    g0 = _run(vrc, w, w.params, pos)
    # the same radiance bits; single scattering's derivatives the same up to the rounding of the
    # other kernel build's instruction schedule (a few ulp per cell term, amplified by the
    # record's cancellation, kappa up to ~150); multiple scattering's derivatives move
    for k in ("L", "L_ss", "L_ms"):
        assert np.array_equal(g[k], g0[k]), k
    for k in ("grad_ss", "hess_ss"):
        scale = np.abs(g0[k]).max(axis=1, keepdims=True) + 1e-30
        assert np.all(np.abs(g[k] - g0[k]) <= 1e-4 * scale), k
    assert not np.allclose(g["hess_ms"], g0["hess_ms"], rtol=1e-3)
    sel = np.arange(pos.shape[0]) if idx is None else np.asarray(idx)
    ref = oracle_replayed(O, O.OracleScene(w.scene), rp, pos[sel], g, rec_ids=sel, idx=sel)
    st = compare_records(g, ref, idx=sel)
    assert st["worst_L"] <= 1.0 and st["worst_g"] <= 1.0 and st["worst_H"] <= 1.0
    return st


def test_small_workload_every_record(vrc):
    st = _check(vrc, W.config1())
    assert st["n"] == W.config1().positions().shape[0]


def test_mid_workload_sample_of_full_launch(vrc):
    w = W.config2()
    n = w.positions().shape[0]
    st = _check(vrc, w, idx=np.arange(5, n, 16))
    assert st["n"] == len(range(5, n, 16))


def test_more_than_one_light_is_refused(vrc):
    w = W.config1()
    w.scene.lights = list(w.scene.lights) + [PointLight((0.2, 0.8, 0.7), (0.5, 0.5, 0.5))]
    with pytest.raises(vrc.VrcError, match="unsupported"):
        _run(vrc, w, replace(w.params, lo_grad=1), w.positions(8))


def test_other_block_shapes_are_refused_and_256_threads_agree(vrc):
    """The option's kernel is built for 256-, 384- and 512-thread blocks: other explicit launch
    shapes are refused; 256 threads in band chunks give the default launch's records up to
    the order of the sums."""
    w = W.config1()
    rp = replace(w.params, lo_grad=1)
    pos = torch.from_numpy(w.positions()).cuda()
    s = vrc.Scene.from_workload(w.scene)
    ref = to_np(vrc.compute_records(s, pos, rp))
    for t in (128,):
        s.set_tuning(threads=t)
        with pytest.raises(vrc.VrcError, match="unsupported"):
            vrc.compute_records(s, pos, rp)
    s.set_tuning(threads=256, chunk_bands=4)
    g = to_np(vrc.compute_records(s, pos, rp))
    torch.cuda.synchronize()
    for k in ("L", "grad", "hess"):
        scale = np.abs(ref[k]).max(axis=1, keepdims=True) + 1e-30
        assert np.all(np.abs(g[k] - ref[k]) <= 1e-4 * scale), k
