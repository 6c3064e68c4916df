"""The N > 1 path of bench.py on CPU: two gloo ranks, disjoint problem shards, and the weak-scaling
reduction (slowest rank's time, all ranks' converged solves)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, e2e, conv = bench.reduce_over_ranks(10.0 + rank, 50.0 - rank, 100 + rank, dist, "cpu")
    x0 = np.stack([p["x0"] for p in bench.workload("config2", 3, rank)])
    gathered = [None] * world
    dist.all_gather_object(gathered, x0.tolist())
    dist.destroy_process_group()
    out.put((rank, ms, e2e, conv, gathered))


def test_two_gloo_ranks_shard_and_reduce():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, conv, gathered in res:
        assert ms == 11.0 and e2e == 50.0 and conv == 201.0
        a, b = np.array(gathered[0]), np.array(gathered[1])
        assert a.shape == b.shape and not np.any(np.all(a[:, None, :] == b[None, :, :], axis=2))


def test_profiled_traffic_only_for_the_captured_kernel(tmp_path, monkeypatch):
    """bench.py reports the roofline traffic from an ncu capture only while the kernel sources hash
    to the captured version, scaled by node-iterations; otherwise, and for workloads without a
    capture, it reports null."""
    import bench
    sha = bench.kernel_sha()
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "capture.md"
    prof.write_text(f"kernel_sha256: {sha}\ndram_bytes_per_node_iteration: 1000\nproblems_captured: 512\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILES", {"config4": "capture.md"})
    assert bench.profiled_traffic("config4", 2048.0) == 1000.0 * 2048
    assert bench.profiled_traffic("config3", 1024.0) is None
    prof.write_text("kernel_sha256: 0000000000000000\ndram_bytes_per_node_iteration: 1000\n")
    assert bench.profiled_traffic("config4", 2048.0) is None
