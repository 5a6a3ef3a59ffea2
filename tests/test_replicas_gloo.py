"""The N-GPU bench runs independent replicas (the method has no exchange step
on one index): each rank builds from its own seeded shard, the timed region is
bracketed by barriers, and the job time is the maximum over ranks.  This checks
that host-side logic with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # slowest rank decides every timing
        mine = [10.0 + rank, 5.0 - rank, 3.0 * (rank + 1)]
        got = bench.max_over_ranks(mine, world)
        # each rank's shard is its own seeded stream, reproducible
        w = bench.workload(False, n=4000)
        a = bench.make_inputs(w, rank)
        b = bench.make_inputs(w, rank)
        same = all(np.array_equal(a[k], b[k]) for k in a if isinstance(a[k], np.ndarray))
        dig = int(np.bitwise_xor.reduce(a["pts"].reshape(-1).astype(np.int64) * 1000003 + np.arange(a["pts"].size)))
        digs = [None] * world
        dist.all_gather_object(digs, dig)
        dist.barrier()
        out.put((rank, got, same, digs, bench.job_throughput(world, w["n"], got[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_max_and_own_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, same, digs, thr in res:
        assert got == [11.0, 5.0, 6.0]
        assert same
        assert digs[0] != digs[1]  # different shards on different ranks
        assert thr == pytest.approx(2 * 4000 / 11e-3 / 1e6)
