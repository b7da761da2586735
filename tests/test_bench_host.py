"""Host-side logic of the benchmark: the multi-rank aggregation (world size
2 over gloo on CPU), the per-rank shards of one global database, and the
reference arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, work = bench.aggregate(1.0 + rank, [10.0 * (rank + 1), 3.0])
    out[rank] = (t, work[0], work[1])
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # slowest rank's time, summed work, identical on both ranks
    assert out[0] == out[1] == (2.0, 30.0, 6.0)


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.5, [7, 8]) == (2.5, [7.0, 8.0])


def test_rank_shards_partition_one_global_database():
    """Under N ranks each rank generates only its balanced contiguous range of
    one global database; the ranges put together are the one-rank database."""
    sys.path.insert(0, ROOT)
    import bench
    q, whole, s0, n_glob = bench.workload(400, 0, 1)
    assert s0 == 0 and n_glob == 400 and whole.n_mol == 400
    parts = [bench.workload(200, r, 2) for r in range(2)]
    assert parts[0][2] == 0 and parts[1][2] == parts[0][1].n_mol and parts[1][3] == 400
    np.testing.assert_array_equal(parts[0][0].xyz, q.xyz)
    xyz = np.concatenate([p[1].xyz for p in parts])
    np.testing.assert_array_equal(xyz, whole.xyz)
    cnt = np.concatenate([p[1].counts for p in parts])
    np.testing.assert_array_equal(cnt, whole.counts)
    assert abs(parts[0][1].n_mol - parts[1][1].n_mol) < 20  # balanced by work


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-db", "1000",
                          "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "evals/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
