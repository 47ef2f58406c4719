"""Splitting the path across GPUs (one process per GPU, torch.distributed).

Records are independent: a batch of n records is split into contiguous shards, one per
rank, with no communication (each rank builds the scene itself; a record's jitter index
is its global index, so the union of the shards equals the single-GPU result).  A query
needs every record near it, so for queries against one shared cache the ranks exchange
their compact record rows (position, radius, radiance, gradient: 16 floats) with one
all-gather, then each answers its own share of the queries.  Weak scaling (each rank an
independent batch) needs neither.  Timings are reduced with the maximum over ranks.
"""
from __future__ import annotations

from typing import Tuple

COMPACT = ("pos", "radius", "L", "grad")        # 3 + 1 + 3 + 9 = 16 floats per record


def shard(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """(start, count) of rank's contiguous share of n_total items; the first
    n_total % world ranks take one extra item."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def pack_compact(records: dict):
    """[n, 16] float32 rows of the fields queries need."""
    import torch
    n = records["L"].shape[0]
    return torch.cat([records[k].reshape(n, -1) for k in COMPACT], dim=1).contiguous()


def unpack_compact(rows) -> dict:
    out, o = {}, 0
    for k, w in zip(COMPACT, (3, 1, 3, 9)):
        v = rows[:, o:o + w]
        out[k] = (v.reshape(-1) if w == 1 else v).contiguous()
        o += w
    return out


def all_gather_records(records: dict, n_total: int, group=None) -> dict:
    """Every rank receives all ranks' compact rows, in rank order (shards are contiguous,
    so this is global record order)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rows = pack_compact(records)
    counts = [shard(n_total, world, r)[1] for r in range(world)]
    width, cmax = rows.shape[1], max(counts)
    # equal-sized messages: pad every shard to the largest, trim after the exchange
    padded = torch.zeros((cmax, width), dtype=rows.dtype, device=rows.device)
    padded[:rows.shape[0]] = rows
    bufs = [torch.empty((cmax, width), dtype=rows.dtype, device=rows.device) for _ in counts]
    dist.all_gather(bufs, padded, group=group)
    return unpack_compact(torch.cat([b[:c] for b, c in zip(bufs, counts)], dim=0))


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
