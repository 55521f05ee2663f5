"""Host logic of the benchmark's multi-rank path on CPU (gloo, world size 2):
the whole-job time is the slowest rank's, the voxel-iterations are summed, and
only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r took 10 (r + 1) ms for 1000 (r + 1) voxel-iterations
        ms, vi = bench._aggregate(dist, 10.0 * (rank + 1), 1000 * (rank + 1), "cpu")
        out.put((rank, ms, vi))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the summed work
    assert res == [(0, 20.0, 3000.0), (1, 20.0, 3000.0)]


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._aggregate(None, 12.5, 7, "cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        n, steps, warmup = 0, 1, 0
    # rank 1 returns at once, without touching the oracle or the workload
    assert bench.run_reference(A()) == 0


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
