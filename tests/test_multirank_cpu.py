"""The bench's N > 1 path runs independent replicas (no data-path collective);
its only collectives are the barrier and the max-over-ranks of the timings.
Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1000.0 + 500.0 * rank, 7.0 - rank]      # per-rank timings (ms)
    got = bench.reduce_max(local, dist, "cpu")
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks_and_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [1500.0, 7.0]
    import bench
    # 2 ranks x 5 steps done in the slowest rank's 1500 ms
    assert abs(bench.job_value(1500.0, 5, 2) - 0.15) < 1e-15
    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
