"""Splitting the path across GPUs (one process per GPU, torch.distributed).

Records are independent: a batch of n records is split into contiguous shards, one per
rank, with no communication (each rank builds the scene itself; a record's jitter index
is its global index, so the union of the shards equals the single-GPU result).  A query
needs every record near it, so for queries against one shared cache the ranks exchange
their compact record rows (position, radius, radiance, gradient: 16 floats; plus the
Hessian, 18 floats, for second-order queries, and the ellipsoid's radii and axes, 12
floats, for ellipsoidal records) with one all-gather; the queries are then split into
contiguous tiles, one per rank, each rank answers its tile, and a second all-gather
returns every answer to every rank.  Weak scaling (each rank an independent batch) needs
neither.  Timings are reduced with the maximum over ranks.
"""
from __future__ import annotations

from typing import Callable, Tuple

COMPACT = ("pos", "radius", "L", "grad")        # 3 + 1 + 3 + 9 = 16 floats per record
WIDTH = {"pos": 3, "radius": 1, "L": 3, "grad": 9, "hess": 18, "radii": 3, "axes": 9}


def compact_fields(extrap_order: int = 1, aniso: bool = False) -> Tuple[str, ...]:
    """The record fields a query needs: Eq. radianceTaylor's position, radius, radiance and
    gradient, the Hessian for second order, the ellipsoid for ellipsoidal records."""
    return COMPACT + (("hess",) if extrap_order == 2 else ()) + (("radii", "axes") if aniso else ())


def shard(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """(start, count) of rank's contiguous share of n_total items; the first
    n_total % world ranks take one extra item."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def pack_compact(records: dict, fields=COMPACT):
    """[n, width] rows of the given fields (float32 on the GPU path)."""
    import torch
    n = records["L"].shape[0]
    return torch.cat([records[k].reshape(n, -1) for k in fields], dim=1).contiguous()


def unpack_compact(rows, fields=COMPACT) -> dict:
    out, o = {}, 0
    for k in fields:
        w = WIDTH[k]
        v = rows[:, o:o + w]
        out[k] = (v.reshape(-1) if w == 1 else v).contiguous()
        o += w
    return out


def _gather_rows(rows, n_total: int, group=None):
    """All ranks' contiguous shares of n_total rows, in rank order, on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    counts = [shard(n_total, world, r)[1] for r in range(world)]
    width, cmax = rows.shape[1], max(counts)
    # equal-sized messages: pad every shard to the largest, trim after the exchange
    padded = torch.zeros((cmax, width), dtype=rows.dtype, device=rows.device)
    padded[:rows.shape[0]] = rows
    bufs = [torch.empty((cmax, width), dtype=rows.dtype, device=rows.device) for _ in counts]
    dist.all_gather(bufs, padded, group=group)
    return torch.cat([b[:c] for b, c in zip(bufs, counts)], dim=0)


def all_gather_records(records: dict, n_total: int, group=None, fields=COMPACT) -> dict:
    """Every rank receives all ranks' compact rows, in rank order (shards are contiguous,
    so this is global record order)."""
    return unpack_compact(_gather_rows(pack_compact(records, fields), n_total, group), fields)


def shared_queries(records: dict, n_total: int, queries, answer: Callable, extrap_order: int = 1,
                   aniso: bool = False, group=None):
    """Queries against one cache whose records are sharded over the ranks.  The compact
    rows (with the Hessian and the ellipsoid where the queries need them) are gathered;
    this rank answers its contiguous tile of `queries` [nq, 3] (the same array on every
    rank) with answer(all_records, tile) -> (rgb [m, 3], count [m]) -- on the GPU a record
    grid and vrc_query_inscatter; then every rank receives every answer, in query order.
    Returns (rgb [nq, 3], count [nq])."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    full = all_gather_records(records, n_total, group, compact_fields(extrap_order, aniso))
    nq = queries.shape[0]
    q0, qn = shard(nq, world, rank)
    rgb, cnt = answer(full, queries[q0:q0 + qn])
    # one exchange for both outputs: the count rides as a float (exact below 2^24)
    rows = torch.cat([rgb.reshape(qn, 3).to(torch.float64), cnt.reshape(qn, 1).to(torch.float64)], dim=1)
    out = _gather_rows(rows.to(queries.device), nq, group)
    return out[:, :3].to(rgb.dtype), out[:, 3].round().to(cnt.dtype)


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
