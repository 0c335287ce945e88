"""The multi-GPU path of the benchmark is replicas only: every rank solves its
own instance and the job time is the maximum over ranks.  Checked here with
two gloo ranks on the CPU (no GPU, no solver call)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, device="cpu")
    # the reference arm runs on rank 0 only; other ranks leave without work
    if rank != 0:
        class A:
            warmup = steps = 1
            workload = "tiny2d"
            strategy = "nobl_mid"
            cpu_sample_its = 1
            gpus = world
        assert bench.run_reference(A()) == 0
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == pytest.approx(2.5)


def test_single_process_keeps_its_value():
    import bench
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25
