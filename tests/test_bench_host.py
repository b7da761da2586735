"""Host-side logic of the benchmark: the multi-rank aggregation (world size
2 over gloo on CPU), per-rank database shards, and the reference arm's JSON
line (the FP64 oracle on the host cores)."""
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


def test_rank_shards_differ_and_repeat():
    sys.path.insert(0, ROOT)
    import bench
    q0, d0 = bench.workload(200, 0)
    q1, d1 = bench.workload(200, 1)
    q0b, d0b = bench.workload(200, 0)
    np.testing.assert_array_equal(d0.xyz, d0b.xyz)
    assert d0.n_mol == d1.n_mol == 200
    assert not np.array_equal(d0.counts, d1.counts) or not np.allclose(d0.xyz[:10], d1.xyz[:10])


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-db", "1000",
                          "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "evals/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
