"""Multi-process path of bench.py (no data-path collective): with world_size
2 on the gloo backend, the timed region's duration is the max over ranks and
the whole-job throughput sums the replicas' work; a batch of channels splits
between the ranks with every channel on exactly one rank."""
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


def _batch_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1903_01111_gb300 import batch as B

    specs = B.draw_channels(9, seed=2, nx_range=(30, 60), ny_range=(12, 24), n_cyl=(1, 2), r_range=(2.0, 4.0))
    mine = B.shard(specs, rank, world)
    nf = B.stack(mine).n_fluid
    v = bench.sharded_mlups(dist, torch, nf, 10, [5.0, 8.0][rank])
    out[rank] = (v, nf, [s.nx for s in mine])
    dist.destroy_process_group()


def test_batch_shards_across_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_batch_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    from paper_1903_01111_gb300 import batch as B

    specs = B.draw_channels(9, seed=2, nx_range=(30, 60), ny_range=(12, 24), n_cyl=(1, 2), r_range=(2.0, 4.0))
    total = B.stack(specs).n_fluid
    assert res[0][1] + res[1][1] == total
    assert sorted(res[0][2] + res[1][2]) == sorted(s.nx for s in specs)
    expect = total * 10 / 0.008 / 1e6
    assert abs(res[0][0] - expect) < 1e-9 * expect and abs(res[1][0] - expect) < 1e-9 * expect
