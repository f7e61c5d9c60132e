"""The multi-GPU form of the path on the host: sharding by samples and the whole-job
reduction bench.py does under torchrun, with world_size-2 gloo ranks on the CPU.  The path
shards without a data-path collective (samples are independent problems), so two shards
projected apart equal one batch projected together."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import solve
from paper_2607_00095_b300 import synthetic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_shards_equal_one_batch():
    uh, pr = synthetic.gen_1d(71, 6, 16, 5, "B")
    u, lam, st, _, _ = solve.project_1d("B", 16, 5, pr, uh)
    parts = [solve.project_1d("B", 16, 5, pr[a:b], uh[a:b]) for a, b in ((0, 3), (3, 6))]
    np.testing.assert_array_equal(np.concatenate([q[0] for q in parts]), u)
    np.testing.assert_array_equal(np.concatenate([q[1] for q in parts]), lam)


def test_shard_seeds_distinct():
    seeds = {bench.shard_seed(1001, r, k) for r in range(4) for k in range(8)}
    assert len(seeds) == 32


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank projects its own shard (a tiny one, with the oracle) and times it
        seed = bench.shard_seed(1001, 0, rank)
        uh, pr = synthetic.gen_1d(seed, 2, 16, 4, "B")
        _, _, st, _, _ = solve.project_1d("B", 16, 4, pr, uh, nthreads=1)
        conv = int((st["status"] == 0).sum())
        elapsed = 10.0 + 5.0 * rank                      # a known per-rank time
        t, c = bench.reduce_over_ranks(elapsed, conv, torch.device("cpu"))
        q.put((rank, t, c, conv))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_2_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    total = sum(r[3] for r in res)
    for rank, t, c, _ in res:
        assert t == 15.0                                 # the slowest rank's time
        assert c == total                                # converged samples of all ranks
