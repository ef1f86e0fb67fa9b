"""The multi-rank bench path on CPU: two gloo ranks (127.0.0.1) run the
replica helpers of bench.py -- per-rank pair seeds, the max over ranks of the
step time and the whole-job rate -- with no GPU and no data-path collective."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.replica_env()
    step_ms = 1.0 + 0.5 * r                       # rank 1 is the slower replica
    slowest = bench.max_over_ranks(step_ms, dist, torch.device("cpu"))
    rate = bench.job_rate(1000.0, w, slowest * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, slowest, rate))


def test_two_replicas_reduce_the_step_time_to_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    for _, _, _, slowest, rate in out:
        assert slowest == 1.5                       # both ranks see the slowest rank's time
        assert abs(rate - 2 * 1000.0 / 1.5e-3) < 1e-6
