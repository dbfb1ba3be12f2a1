"""The multi-replica path of bench.py on CPU: two gloo ranks reduce their step times to the
slowest one and report the whole-job throughput; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    slowest = bench.reduce_max(times[rank], dist, "cpu")
    value = bench.job_mpix_per_s(3 * 4096 * 4096, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{slowest!r} {value!r}\n")


def test_two_gloo_ranks_take_the_slowest(tmp_path):
    import torch.multiprocessing as mp
    times = [0.0125, 0.0175]
    mp.start_processes(_rank_main, args=(2, _free_port(), times, str(tmp_path)), nprocs=2, start_method="spawn")
    got = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for slowest, value in got:
        assert float(slowest) == max(times)
        assert float(value) == pytest.approx(2 * 3 * 4096 * 4096 / max(times) / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(0.5, None, "cpu") == 0.5
    assert bench.job_mpix_per_s(1e6, 1, 0.5) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        cpu_rows = 1024
        steps = 1
        warmup = 0
    assert bench.run_reference(Args()) == 0  # returns before touching the oracle or the image
