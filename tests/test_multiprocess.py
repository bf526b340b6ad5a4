"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1), no GPU.

Under torchrun each rank advances its own jobs (replicas of the grid workloads, or its own serving
stream): nothing is exchanged on the data path; the ranks only agree on the timing (max over ranks)
and rank 0 merges the serving statistics.  Checked here: the max reduction, the gather in rank
order, the partition of a job list, and the merged percentiles and throughput."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    try:
        m = bench.dist_max(1.5 + rank)
        recs = bench.gather_objects({"lat": [0.1 * (rank + 1), 0.2 * (rank + 1)], "work": 10.0 * (rank + 1),
                                     "makespan": 2.0 + rank})
        part = bench.shard(list(range(11)), rank, world)
        env = bench.dist_env()
        queue.put((rank, m, recs, part, env))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_gather_shard_and_merge():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, recs0, part0, env0), (r1, m1, recs1, part1, env1) = out
    assert (r0, r1) == (0, 1) and m0 == m1 == 2.5
    assert env0 == (2, 0, 0) and env1 == (2, 1, 1)
    assert recs0 == recs1 and [r["work"] for r in recs0] == [10.0, 20.0]
    assert sorted(part0 + part1) == list(range(11)) and not set(part0) & set(part1)
    sys.path.insert(0, ROOT)
    import bench

    st = bench.merge_serving(recs0)
    assert st["jobs"] == 4 and st["makespan_s"] == 3.0 and st["cell_rk_stage_updates_per_s"] == pytest.approx(10.0)
    assert st["p50_s"] == pytest.approx(np.percentile([0.1, 0.2, 0.2, 0.4], 50))
