"""Multi-process path of bench.py (replicas only: no data-path collective):
with world_size 2 on the gloo backend, the timed region's duration is the
max over ranks and the whole-job throughput sums the replicas' work."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.0, 20.0][rank]
    got = bench._max_over_ranks(dist, torch, ms)
    dist.barrier()
    out[rank] = (got, bench.replica_mlups(world, 1_000_000, 10, got))
    dist.destroy_process_group()


def test_two_replicas_max_time_and_summed_throughput():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # 2 replicas x 1e6 fluid nodes x 10 steps in 20 ms
    assert abs(res[0][1] - 2 * 1e6 * 10 / 0.020 / 1e6) < 1e-9
