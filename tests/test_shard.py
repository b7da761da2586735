"""One database split over ranks: the balanced contiguous partition, and the
gather and per-query top-k merge on rank 0, run as two gloo ranks on CPU on
host arrays (the screen's own equivalence under sharding -- global stream
keys -- is a GPU test, test_gpu_parity.test_sharded_screen_reproduces_the_full_screen)."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2607_20766_b300 import shard  # noqa: E402


@pytest.mark.parametrize("n_ranks", [1, 2, 3, 8])
def test_partition_is_contiguous_and_balanced(n_ranks):
    rng = np.random.default_rng(n_ranks)
    nd = rng.integers(18, 61, 1001)
    nq = rng.integers(20, 49, 5)
    parts = shard.partition(nd, nq, n_ranks)
    assert parts[0][0] == 0 and parts[-1][1] == len(nd)
    assert all(parts[r][1] == parts[r + 1][0] for r in range(n_ranks - 1))
    cost = len(nq) * nd + nq.sum()
    work = [cost[s:e].sum() for s, e in parts]
    # each cut is off the ideal share by at most one molecule's cost
    assert max(work) - min(work) <= 2 * cost.max()
    assert sum(work) == cost.sum()


def test_partition_of_a_tiny_database_leaves_empty_ranges():
    parts = shard.partition([30, 40], [25], 4)
    assert parts[0][0] == 0 and parts[-1][1] == 2
    assert sum(e - s for s, e in parts) == 2


def _global_results(n_q, n_global):
    rng = np.random.default_rng(7)
    # quantised values so that ties occur (merge order must not depend on the split)
    T = np.round(rng.uniform(0, 1, (n_q, n_global)), 2).astype(np.float32)
    seT = rng.uniform(0, 0.01, (n_q, n_global, 2)).astype(np.float32)
    nu = rng.integers(1, 64, (n_q, n_global)).astype(np.int32) * 256
    return T, seT, nu


def _rank(rank, world, port, parts, n_q, n_global, k, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2607_20766_b300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T, seT, nu = _global_results(n_q, n_global)
    s, e = parts[rank]
    # the local screen's pair order: q * n_local + d_local
    loc_T = torch.tensor(T[:, s:e].reshape(-1))
    loc_se = torch.tensor(seT[:, s:e].reshape(-1, 2))
    loc_nu = torch.tensor(nu[:, s:e].reshape(-1))
    gT = S.gather_screen(loc_T, s, e, n_q, n_global)
    gse = S.gather_screen(loc_se, s, e, n_q, n_global)
    gnu = S.gather_screen(loc_nu, s, e, n_q, n_global)
    top = S.topk_merge(loc_T, s, n_q, k)
    if rank == 0:
        out["T"] = gT.numpy()
        out["se"] = gse.numpy()
        out["nu"] = gnu.numpy()
        out["top_v"] = top[0].numpy()
        out["top_i"] = top[1].numpy()
    else:
        out[f"none{rank}"] = (gT is None and gse is None and gnu is None and top is None)
    dist.destroy_process_group()


@pytest.mark.parametrize("uneven", [False, True])
def test_gather_and_topk_merge_over_two_gloo_ranks(uneven):
    n_q, n_global, k = 3, 101, 10
    parts = [(0, 30), (30, 101)] if uneven else shard.partition(np.full(n_global, 40), [30] * n_q, 2)
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29600 + (os.getpid() + 17 * uneven) % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, parts, n_q, n_global, k, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    T, seT, nu = _global_results(n_q, n_global)
    np.testing.assert_array_equal(out["T"], T.reshape(-1))
    np.testing.assert_array_equal(out["se"], seT.reshape(-1, 2))
    np.testing.assert_array_equal(out["nu"], nu.reshape(-1))
    assert out["none1"]
    for q in range(n_q):
        order = np.lexsort((np.arange(n_global), -T[q].astype(np.float64)))[:k]  # value desc, id asc
        np.testing.assert_array_equal(out["top_i"][q], order)
        np.testing.assert_array_equal(out["top_v"][q], T[q, order])


def test_local_topk_breaks_ties_by_id():
    T = torch.tensor([0.5, 0.9, 0.5, 0.9, 0.1, 0.5], dtype=torch.float32)
    v, i = shard.local_topk(T, start=100, n_q=2, k=2)
    np.testing.assert_array_equal(i.numpy(), [[101, 100], [100, 102]])
    np.testing.assert_array_equal(v.numpy(), np.float32([[0.9, 0.5], [0.9, 0.5]]))
