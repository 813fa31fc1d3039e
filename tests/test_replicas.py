"""The multi-process form of bench.py (replicas only: the path has no exchange step on one
node here, so N ranks run N independent copies of the workload) as world-size-2 gloo ranks
on the CPU: every rank reports the job time as the slowest rank's and the whole-job
throughput as N x units / that time."""
import os
import sys
import tempfile

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.replica_throughput(10.0 * (rank + 1), 100.0, world, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(f"{ms} {value}\n")
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(2, port, d), nprocs=2, join=True, start_method="spawn")
        for r in range(2):
            ms, value = map(float, open(os.path.join(d, f"r{r}.txt")).read().split())
            assert ms == 20.0                      # the slower rank's time
            assert value == pytest.approx(2 * 100.0 / 0.020)


def test_replica_throughput_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_throughput(4.0, 8.0, 1)
    assert ms == 4.0 and value == pytest.approx(2000.0)
