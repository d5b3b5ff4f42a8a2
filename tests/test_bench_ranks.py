"""The multi-rank (replicas) timing of bench.py on CPU: two gloo ranks, each with its own elapsed
time, agree on the whole-job throughput = all units / the slowest rank's time."""
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


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, max_s = bench.job_throughput(1.0 + rank, 10, world)   # rank r took 1 + r seconds
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{value} {max_s}\n")
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        value, max_s = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert max_s == 2.0 and value == 2 * 10 / 2.0


def test_single_replica_needs_no_process_group():
    import bench
    assert bench.job_throughput(0.5, 32, 1) == (64.0, 0.5)
