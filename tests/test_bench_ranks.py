"""Multi-rank path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job's time is the slowest rank's and its updates the sum."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_ranks(1.0 + rank, 1000 * (rank + 1), device="cpu")
    r, w = bench._dist()
    out.put((rank, t, u, r, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, u, r, w in res:
        assert t == 2.0 and u == 3000.0      # max time over ranks, sum of updates
        assert r == rank and w == 2


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(1.5, 42) == (1.5, 42.0)


def test_traffic_figure_is_read_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the
    kernel code hash matches the one the counters were taken on."""
    import bench
    prof = tmp_path / "prof.md"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", "prof.md")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [])
    prof.write_text(f"# x\n\n- kernel_sha256: `{bench.kernel_hash()}` (comment-free code)\n"
                    "- dram_bytes_per_vehicle_update: `123.5`\n")
    assert bench.measured_traffic_per_update() == 123.5
    prof.write_text("- kernel_sha256: `0000000000000000`\n- dram_bytes_per_vehicle_update: `123.5`\n")
    assert bench.measured_traffic_per_update() is None


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cuh"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cuh"])
    src.write_text("int f() { return 1; }  // one\n")
    h1 = bench.kernel_hash()
    src.write_text("// a comment\nint f() { return 1; }  // two\n\n")
    assert bench.kernel_hash() == h1
    src.write_text("int f() { return 2; }\n")
    assert bench.kernel_hash() != h1
