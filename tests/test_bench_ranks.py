"""Multi-rank logic of bench.py on CPU: two gloo ranks, each a replica with
its own step time; the job reports the max step time and the summed
throughput (replicas only: no collective on the data path)."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1.0 + rank          # rank 1 is slower
    ms = bench.max_over_ranks(local_ms, world)
    q.put((rank, ms, bench.job_value(1000, ms, world), bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env in out:
        assert ms == 2.0                      # the slowest rank's time
        assert value == 1000 * 2 / 2.0e-3     # both replicas' work over that time
        assert env[0] == rank and env[1] == 2
