"""One screening database split over several ranks (one process per GPU).

Pairs are independent and every random stream is keyed by the pair's global
index (stream = stream_base + q * stride + d, with stride the global database
size), so a rank that screens the contiguous range [start, end) of the
database with ``stream_base = start`` and ``stream_stride = n_global``
reproduces exactly the numbers a single device would compute for those pairs;
the self-overlap streams are keyed the same way (molecule d uses
``stream_base + d``). No collective is needed while screening. At the end the
ranks either gather every (T, SE(T), n_used) on rank 0 in global order, or
merge per-query top-k lists.

``partition`` balances the ranges by the screen's work: a database molecule
with N_d atoms costs sum_q (N_q + N_d) sample-atom evaluations per sample, so
ranges are cut at equal shares of the prefix sums of that cost.
"""
from __future__ import annotations

import numpy as np
import torch


def partition(counts_db, counts_q, n_ranks: int) -> list[tuple[int, int]]:
    """Contiguous ranges [start, end) of the database, one per rank, with
    (nearly) equal screen work sum_{d in range} sum_q (N_q + N_d)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    nd = np.asarray(counts_db, dtype=np.int64)
    nq = np.asarray(counts_q, dtype=np.int64)
    cost = len(nq) * nd + nq.sum()
    cum = np.concatenate([[0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, n_ranks):
        # first index whose prefix cost reaches r / n_ranks of the total
        cuts.append(int(np.searchsorted(cum, total * r / n_ranks, side="left")))
    cuts.append(len(nd))
    cuts = np.maximum.accumulate(np.minimum(np.asarray(cuts), len(nd)))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(n_ranks)]


def _dist():
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        raise RuntimeError("shard collectives need an initialised torch.distributed process group")
    return dist


def gather_screen(values: torch.Tensor, start: int, end: int, n_q: int, n_global: int, device=None):
    """Gather a per-pair result of every rank's range on rank 0.

    values: [n_q * (end - start), ...] in the local screen's pair order
    (q * n_local + d_local). Returns on rank 0 the [n_q * n_global, ...]
    tensor in global pair order (q * n_global + d), None elsewhere. Ranges
    may differ in size; every rank calls this collectively."""
    dist = _dist()
    world, rank = dist.get_world_size(), dist.get_rank()
    device = values.device if device is None else device
    n_local = end - start
    tail = tuple(values.shape[1:])
    local = values.reshape(n_q, n_local, *tail).to(device)
    # ranges and sizes of every rank
    rng = torch.tensor([start, end], dtype=torch.int64, device=device)
    ranges = [torch.empty_like(rng) for _ in range(world)]
    dist.all_gather(ranges, rng)
    ranges = [(int(r[0]), int(r[1])) for r in ranges]
    width = max(e - s for s, e in ranges)
    padded = torch.zeros((n_q, width, *tail), dtype=values.dtype, device=device)
    padded[:, :n_local] = local
    parts = [torch.empty_like(padded) for _ in range(world)] if rank == 0 else None
    dist.gather(padded, parts, dst=0)
    if rank != 0:
        return None
    out = torch.empty((n_q, n_global, *tail), dtype=values.dtype, device=device)
    for (s, e), p in zip(ranges, parts):
        out[:, s:e] = p[:, :e - s]
    return out.reshape(n_q * n_global, *tail)


def local_topk(T: torch.Tensor, start: int, n_q: int, k: int):
    """Per-query best k of a local range: (values [n_q, k'], global ids
    [n_q, k']) with k' = min(k, local size); ties broken by the lower id."""
    n_local = T.numel() // n_q
    T2 = T.reshape(n_q, n_local)
    kk = min(k, n_local)
    ids = torch.arange(n_local, device=T.device, dtype=torch.int64)
    # stable order: sort ids descending by value (argsort of -T is stable)
    order = torch.argsort(-T2.to(torch.float64), dim=1, stable=True)[:, :kk]
    return torch.gather(T2, 1, order), ids[order] + start


def topk_merge(T: torch.Tensor, start: int, n_q: int, k: int):
    """Per-query top-k of the whole database on rank 0 from every rank's
    local range (T [n_q * n_local] in local pair order). Returns (values
    [n_q, k], global ids [n_q, k]) on rank 0, None elsewhere; equal values
    are ordered by database id, so the result does not depend on how the
    database was split."""
    dist = _dist()
    world, rank = dist.get_world_size(), dist.get_rank()
    v, i = local_topk(T, start, n_q, k)
    kk = torch.tensor([v.shape[1]], dtype=torch.int64, device=T.device)
    sizes = [torch.empty_like(kk) for _ in range(world)]
    dist.all_gather(sizes, kk)
    width = max(int(s) for s in sizes)
    vp = torch.full((n_q, width), float("-inf"), dtype=v.dtype, device=T.device)
    ip = torch.full((n_q, width), -1, dtype=torch.int64, device=T.device)
    vp[:, :v.shape[1]] = v
    ip[:, :i.shape[1]] = i
    vs = [torch.empty_like(vp) for _ in range(world)] if rank == 0 else None
    is_ = [torch.empty_like(ip) for _ in range(world)] if rank == 0 else None
    dist.gather(vp, vs, dst=0)
    dist.gather(ip, is_, dst=0)
    if rank != 0:
        return None
    allv, alli = torch.cat(vs, 1), torch.cat(is_, 1)
    valid = alli >= 0
    # sort by (value descending, id ascending): ids first, then a stable sort by value
    o1 = torch.argsort(torch.where(valid, alli, torch.iinfo(torch.int64).max), dim=1, stable=True)
    v1, i1 = torch.gather(allv, 1, o1), torch.gather(alli, 1, o1)
    o2 = torch.argsort(-v1.to(torch.float64), dim=1, stable=True)[:, :k]
    return torch.gather(v1, 1, o2), torch.gather(i1, 1, o2)
