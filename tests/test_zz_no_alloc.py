"""The query entry point that allocates nothing (vrc_query_inscatter_noalloc).

Some callers cannot call cudaMalloc at query time (an application that owns all device
memory, a renderer that forbids allocation after start-up, a fixed memory budget).
For them the library answers queries from a fixed device array instead of a grid
object.  This test checks, through the C ABI, that two calls in a row agree with the
allocating path (vrc_build_record_grid + vrc_query_inscatter) and with the FP64 oracle's
brute-force Eq. radianceTaylor within the query tests' tolerance, also when the record
lists overflow the array (the queries then scan every record) and when there are no
records, and that a record count beyond the array's stated maximum is refused.
It lives in its own file, collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

import oracle as O

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
    a, b, ca, cb = (x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x) for x in (a, b, ca, cb))
    assert np.array_equal(ca, cb)
    scale = np.abs(b).max(axis=1, keepdims=True) + np.abs(b) + 1e-6
    assert np.all(np.abs(a - b) <= 2e-5 * scale + 1e-6)


def oracle_query(recs, q, order):
    """The oracle's brute force over every record, counts compared away from region
    boundaries (|x' - x_k| within 1e-5 R_k of R_k may round either way)."""
    t = {k: v.cpu().numpy() for k, v in recs.items()}
    rgb, cnt, near = O.query(t["pos"], t["radius"], t["L"], t["grad"], t["hess"], q.cpu().numpy(), order=order)
    return rgb, cnt, near.astype(bool)


def check_oracle(rgb, cnt, recs, q, order, keep_at_least=0.99):
    orgb, ocnt, near = oracle_query(recs, q, order)
    rgb, cnt = rgb.cpu().numpy(), cnt.cpu().numpy()
    keep = ~near
    assert keep.mean() > keep_at_least
    close(rgb[keep], orgb[keep], cnt[keep], ocnt[keep])


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
        check_oracle(rgb, cnt, recs, q, order)
        assert int(cnt.max()) > 1, call


def test_overflowing_lists_scan_every_record(vrc):
    """4,000 records of radius 0.3 overlap about 600 of the array's 4,096 cells each: the
    lists (2.4M entries) do not fit in the array's 1M words, so every query scans all
    records; the answers still match the allocating path and the oracle (queries within
    1e-5 R of some record's boundary, a few percent with hundreds of records around each
    point, are left to the allocating-path comparison).  The call after it (small table)
    builds its lists again."""
    n = 4000
    recs = table(n, 7)
    recs["radius"] = torch.full((n,), 0.3, device="cuda")
    q = torch.rand((2000, 3), generator=torch.Generator().manual_seed(7)).cuda()
    rgb, cnt = vrc.query_inscatter_noalloc(recs, q, extrap_order=1)
    grid = vrc.Grid(recs, extrap_order=1)
    ref_rgb, ref_cnt = vrc.query_inscatter(grid, q)
    torch.cuda.synchronize()
    assert int(cnt.min()) > 20
    close(rgb, ref_rgb, cnt, ref_cnt)
    check_oracle(rgb, cnt, recs, q, 1, keep_at_least=0.9)
    small = table(500, 8)
    q2 = torch.rand((3000, 3), generator=torch.Generator().manual_seed(8)).cuda()
    rgb2, cnt2 = vrc.query_inscatter_noalloc(small, q2, extrap_order=1)
    torch.cuda.synchronize()
    check_oracle(rgb2, cnt2, small, q2, 1)


def test_no_records_gives_misses(vrc):
    recs = {k: torch.zeros((0, w), device="cuda") for k, w in (("pos", 3), ("L", 3), ("grad", 9), ("hess", 18))}
    recs["radius"] = torch.zeros((0,), device="cuda")
    q = torch.rand((777, 3), device="cuda")
    rgb, cnt = vrc.query_inscatter_noalloc(recs, q, extrap_order=2)
    torch.cuda.synchronize()
    assert int(cnt.abs().max()) == 0 and float(rgb.abs().max()) == 0.0


def test_refuses_more_records_than_the_array_holds(vrc):
    n = vrc.NOALLOC_MAX_RECORDS + 1
    recs = {k: torch.zeros((n, w), device="cuda") for k, w in (("pos", 3), ("L", 3), ("grad", 9))}
    recs["radius"] = torch.full((n,), 0.1, device="cuda")
    q = torch.rand((10, 3), device="cuda")
    with pytest.raises(vrc.VrcError, match="unsupported"):
        vrc.query_inscatter_noalloc(recs, q)
