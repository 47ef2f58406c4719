"""Multi-rank logic on CPU: world size 2 with the gloo backend (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_09258_gb300.sharding import all_gather_records, max_over_ranks, shard


def test_shards_partition_every_size():
    for n in (0, 1, 5, 7, 4096, 100001):
        for world in (1, 2, 3, 8):
            spans = [shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (s0, c0), (s1, _) in zip(spans, spans[1:]):
                assert s0 + c0 == s1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_total, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, count = shard(n_total, world, rank)
    # each rank's records: values that encode the global record index
    idx = torch.arange(start, start + count, dtype=torch.float32)
    rec = {"pos": idx[:, None].repeat(1, 3), "radius": idx + 0.5, "L": idx[:, None].repeat(1, 3) * 2,
           "grad": idx[:, None].repeat(1, 9) * 3}
    full = all_gather_records(rec, n_total)
    ok = bool(torch.equal(full["radius"], torch.arange(n_total, dtype=torch.float32) + 0.5)) and \
        full["grad"].shape == (n_total, 9) and bool(torch.equal(full["L"][:, 1], torch.arange(n_total).float() * 2))
    t = max_over_ranks(1.0 + rank)
    q.put((rank, ok, t))
    dist.destroy_process_group()


@pytest.mark.parametrize("n_total", [7, 4096])
def test_all_gather_and_max_over_two_gloo_ranks(n_total):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_total, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, t in res:
        assert ok, rank
        assert t == 2.0


def _oracle_shard(rank, world, n_total):
    """This rank's records of the small workload (the FP64 oracle stands in for the record
    kernel on CPU; jitter indices are global, so the shards' union is the one-rank set)."""
    import numpy as np
    import oracle as O
    import workloads as W
    w = W.config1()
    pos = w.positions(n_total)
    start, count = shard(n_total, world, rank)
    ids = np.arange(start, start + count)
    r = O.records(O.OracleScene(w.scene), w.params, pos[ids], rec_ids=ids, n_threads=1)
    radii, axes, _, _, _ = O.aniso_records(r["L"], r["hess"], w.params.eps, w.params.r_min, w.params.r_max)
    rec = {"pos": pos[ids], "radius": r["radius"], "L": r["L"], "grad": r["grad"], "hess": r["hess"],
           "radii": radii, "axes": axes.reshape(-1, 9)}
    return {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)) for k, v in rec.items()}, w


def _answer(order, aniso):
    """Eq. radianceTaylor over the gathered table (the oracle's brute force on CPU)."""
    def f(full, tile):
        import numpy as np
        import oracle as O
        t = {k: v.numpy() for k, v in full.items()}
        hess = t.get("hess")
        if aniso:
            radii, axes = t["radii"].astype(np.float64), t["axes"].reshape(-1, 3, 3).astype(np.float64)
            M = np.einsum("nik,ni,nil->nkl", axes, 1.0 / radii ** 2, axes)
            m6 = M[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
            rgb, cnt, _ = O.query_aniso(t["pos"], m6, t["L"], t["grad"], hess, tile.numpy(), order=order)
        else:
            rgb, cnt, _ = O.query(t["pos"], t["radius"], t["L"], t["grad"], hess, tile.numpy(), order=order)
        return torch.from_numpy(rgb), torch.from_numpy(cnt)
    return f


def _query_worker(rank, world, port, n_total, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1805_09258_gb300.sharding import shared_queries
    rec, w = _oracle_shard(rank, world, n_total)
    queries = torch.from_numpy(w.queries(301))
    out = {}
    for order, aniso in ((1, False), (2, False), (1, True)):
        rgb, cnt = shared_queries(rec, n_total, queries, _answer(order, aniso), extrap_order=order, aniso=aniso)
        out[(order, aniso)] = (rgb.numpy(), cnt.numpy())
    q.put((rank, out))
    dist.destroy_process_group()


def test_shared_queries_over_two_gloo_ranks_equal_one_rank():
    """Records sharded over two ranks, their rows gathered (with the Hessian for order 2 and
    the ellipsoid for ellipsoidal records), the queries split into one tile per rank and
    the answers gathered: every rank holds, bit for bit, the one-rank answer."""
    import numpy as np
    n_total = 45
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_query_worker, args=(r, 2, port, n_total, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rec, w = _oracle_shard(0, 1, n_total)
    queries = torch.from_numpy(w.queries(301))
    for key in ((1, False), (2, False), (1, True)):
        rgb1, cnt1 = _answer(*key)(rec, queries)
        for rank in (0, 1):
            rgb, cnt = res[rank][key]
            assert np.array_equal(rgb, rgb1.numpy().astype(rgb.dtype)) and np.array_equal(cnt, cnt1.numpy()), key
        assert (cnt1.numpy() > 0).mean() > 0.3
