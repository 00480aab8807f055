"""Host logic of bench.py that runs without a GPU: the replicas' max / sum reductions over gloo
ranks, and the DRAM-traffic lookup in profiles/traffic.md."""
import os
import socket

import pytest


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = (bench._gather_max(dist, 1.5 + rank), bench._gather_sum(dist, 10 * (rank + 1)))
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reductions_over_gloo():
    import multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == (2.5, 30.0)


def test_reductions_without_a_process_group_are_identity():
    import bench
    assert bench._gather_max(None, 3.25) == 3.25
    assert bench._gather_sum(None, 7) == 7


def test_traffic_lookup(tmp_path, monkeypatch):
    import bench
    src_dir = tmp_path / "paper_1207_0486_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "k.cu").write_text("// kernel\n")
    import hashlib
    digest = hashlib.sha256(b"// kernel\n").hexdigest()[:12]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.md").write_text(
        "| kernel | bytes | file | sha |\n|---|---|---|---|\n"
        f"| `k_a` | 1234 | k.cu | {digest} |\n| `k_b` | 99 | k.cu | 000000000000 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k_a") == 1234
    assert bench.dram_traffic("k_b") is None   # source changed since the capture
    assert bench.dram_traffic("k_c") is None   # not captured
