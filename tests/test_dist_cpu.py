"""Multi-process plumbing of bench.py (replicas: barrier and max over ranks,
no collective on the data path), run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    out[rank] = bench.max_over_ranks(w, 1.5 + rank)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_max_time():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_prints_only_on_rank_zero(capsys):
    import bench

    class A:
        workload = "tiny_64_coplanar"
        steps = 1
        warmup = 0
        gpus = 2

    bench.run_reference(A(), world=2, rank=1)
    assert capsys.readouterr().out == ""
