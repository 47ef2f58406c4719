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
