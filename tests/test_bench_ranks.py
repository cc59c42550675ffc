"""Host logic of the benchmark's replica runs (N > 1 ranks): two gloo ranks on the CPU.

The solve does not shard (each rank solves its own replica), so the only cross-rank step is the
aggregation: the job time is the slowest rank's, the pushed links and kernel launches are
summed. Run as real processes with torch.distributed (gloo, 127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (10 + 5 r) ms, pushed (1 + r) G links, launched (100 + r) kernels
    res = bench.aggregate(dist, 10.0 + 5 * rank, (1 + rank) * 1e9, 100 + rank)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total_ms, pushed, launches = res[r]
        assert total_ms == 15.0                 # slowest rank
        assert pushed == 3e9 and launches == 201
    # the whole-job rate is summed work over the slowest time
    assert res[0][1] / (res[0][0] * 1e-3) / 1e9 == pytest.approx(200.0)


def test_aggregation_without_process_group_is_identity():
    import bench
    assert bench.aggregate(None, 12.5, 7.0, 3) == (12.5, 7.0, 3)
