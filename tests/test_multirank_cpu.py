"""The N-GPU bench path on the CPU (no GPU): one independent replica per rank,
no collective on the data path, the job's throughput from the slowest rank's
time and every rank's bytes.  Two gloo ranks over 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
    dist.barrier()
    q.put((rank, t, u))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_aggregation_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, u in res:
        assert t == 15.0             # the slowest rank's time
        assert u == 3000.0           # bytes of every rank


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_over_ranks(3.0, 7.0, 1) == (3.0, 7.0)
