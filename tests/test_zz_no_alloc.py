"""The query entry point that allocates nothing (vrc_query_inscatter_noalloc).

Some callers cannot call cudaMalloc at query time (an application that owns all device
memory, a renderer that forbids allocation after start-up, a fixed memory budget).
For them the library answers queries from a fixed device array instead of a grid
object.  This test checks, through the C ABI, that two calls in a row agree with the
allocating path (vrc_build_record_grid + vrc_query_inscatter) within the query tests'
tolerance, and that a record count beyond the array's stated maximum is refused.
It lives in its own file, collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

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


def table(n, seed):
    rng = np.random.default_rng(seed)
    t = dict(pos=rng.uniform(0, 1, (n, 3)), radius=rng.uniform(0.03, 0.3, n), L=rng.uniform(0.05, 1, (n, 3)),
             grad=rng.normal(size=(n, 9)) * 0.5, hess=rng.normal(size=(n, 18)) * 2.0)
    return {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in t.items()}


def close(a, b, ca, cb):
    a, b, ca, cb = (x.cpu().numpy() for x in (a, b, ca, cb))
    assert np.array_equal(ca, cb)
    scale = np.abs(b).max(axis=1, keepdims=True) + np.abs(b) + 1e-6
    assert np.all(np.abs(a - b) <= 2e-5 * scale + 1e-6)


@pytest.mark.parametrize("order", [1, 2])
def test_two_calls_match_the_allocating_path(vrc, order):
    for call, (n, nq, seed) in enumerate(((700, 30000, 1), (1500, 12345, 2))):
        recs = table(n, seed)
        q = torch.rand((nq, 3), generator=torch.Generator().manual_seed(seed)).cuda()
        grid = vrc.Grid(recs, extrap_order=order)
        ref_rgb, ref_cnt = vrc.query_inscatter(grid, q)
        rgb, cnt = vrc.query_inscatter_noalloc(recs, q, extrap_order=order)
        torch.cuda.synchronize()
        close(rgb, ref_rgb, cnt, ref_cnt)
        assert int(cnt.max()) > 1, call


def test_refuses_more_records_than_the_array_holds(vrc):
    n = vrc.NOALLOC_MAX_RECORDS + 1
    recs = {k: torch.zeros((n, w), device="cuda") for k, w in (("pos", 3), ("L", 3), ("grad", 9))}
    recs["radius"] = torch.full((n,), 0.1, device="cuda")
    q = torch.rand((10, 3), device="cuda")
    with pytest.raises(vrc.VrcError, match="unsupported"):
        vrc.query_inscatter_noalloc(recs, q)
