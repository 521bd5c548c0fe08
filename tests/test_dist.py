"""The multi-process (N > 1) path of bench.py on CPU: two gloo ranks meet at the
barrier, agree on the slowest rank's time and report the whole-job figure.
(On GPUs the same code runs with NCCL, one rank per GPU, replicas only.)"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), MPC_BENCH_BACKEND="gloo")
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init()
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 * (r + 1), w)      # rank r "took" 10 (r+1) ms
    v = bench.job_throughput(1_000_000_000, 5, w, t)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, t, v))


@pytest.mark.parametrize("world", [2])
def test_two_rank_replicas(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == list(range(world))
    for r, w, t, v in out:
        assert w == world
        assert t == 10.0 * world          # max over ranks
        # world x 1e9 MACs x 5 steps in 20 ms
        assert abs(v - world * 1e9 * 5 / 0.020 / 1e9) < 1e-6


def test_job_throughput_single_rank():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert abs(bench.job_throughput(2_000_000_000, 10, 1, 1000.0) - 20.0) < 1e-9
