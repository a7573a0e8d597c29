"""Multi-GPU path of bench.py on CPU: world size 2 over gloo.

The path has no data exchange between cases, so N GPUs run N independent replicas of the workload; the only
collective is the reduction of the step time (max over ranks) and the barrier around the timed region.  This
checks that reduction and the job throughput built from it, with ranks that report different times."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.slowest_rank_ms(10.0 + 2.5 * rank, dist, "cpu")
    out[rank] = (ms, bench.job_updates_per_s(1_000_000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_value_counts_all_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == pytest.approx(12.5)
        assert value == pytest.approx(2 * 1_000_000 / 12.5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(7.0, None, "cpu") == 7.0
    assert bench.job_updates_per_s(100, 1, 2.0) == pytest.approx(5e4)


def test_clock_sampler_follows_cuda_visible_devices(monkeypatch):
    import bench
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    assert bench.smi_device(0) == "3" and bench.smi_device(1) == "5"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1a2b")
    assert bench.smi_device(0) == "GPU-1a2b"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.smi_device(2) == "2"
