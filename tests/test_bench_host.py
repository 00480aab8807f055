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
    (src_dir / "k.cu").write_text("// kernels\n__global__ void k_a(int x) {\n  if (x) { x = 1; }\n}\n"
                                  "__device__ int helper(int y) { return y; }\n")
    digest = bench.kernel_source_hash(str(src_dir / "k.cu"), ["k_a", "helper"])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.md").write_text(
        "| kernel | bytes | file | functions | sha |\n|---|---|---|---|---|\n"
        f"| `k_a` | 1234 | k.cu | `k_a`, `helper` | {digest} |\n| `k_b` | 99 | k.cu | `k_a` | 000000000000 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k_a") == 1234
    assert bench.dram_traffic("k_b") is None   # source changed since the capture
    assert bench.dram_traffic("k_c") is None   # not captured
    # an edit elsewhere in the file keeps the figure; an edit inside a listed function drops it
    (src_dir / "k.cu").write_text("// kernels, edited comment\n__global__ void k_a(int x) {\n  if (x) { x = 1; }\n}\n"
                                  "__device__ int helper(int y) { return y; }\n")
    assert bench.dram_traffic("k_a") == 1234
    (src_dir / "k.cu").write_text("__global__ void k_a(int x) {\n  if (x) { x = 2; }\n}\n"
                                  "__device__ int helper(int y) { return y; }\n")
    assert bench.dram_traffic("k_a") is None


def test_roofline_of_dominant_class():
    import bench
    n = 5_389_312
    # SpMV dominant: FP64-pipe bound, reported against the derived FP64 peak
    kt = {0: (825.0, 4988), 1: (16.5, 316), 2: (171.0, 5304), 3: (191.7, 5056), 4: (800.0, 4672)}
    r = bench.roofline_of(kt, n, 1, 2098.0, 6791.0, "measured", 2070.0)
    assert r["bound"] == "alu" and r["kernel"] == "k_cg_spmv" and r["unit"] == "TFLOP/s"
    pk = bench.fp64_peak_tflops(2070.0)
    assert abs(pk - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-9
    t = 825.0e-3 / 4988
    assert abs(r["achieved"] - round(32 * n / t / 1e12, 4)) < 1e-9
    assert abs(r["hbm_equivalent"]["achieved"] - round(136 * n / t / 1e9, 1)) < 1e-9
    assert 0.6 < r["hbm_equivalent"]["frac"] < 0.7 and 0.75 < r["frac"] < 0.9
    assert set(r["classes"]) == set(bench.KT_NAMES)
    # fused line dominant: HBM
    kt[4] = (900.0, 4672)
    r = bench.roofline_of(kt, n, 1, 2098.0, 6791.0, "measured", None)
    assert r["bound"] == "hbm" and r["kernel"] == "k_update_line" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - round(88 * n / (900e-3 / 4672) / 1e9, 1)) < 1e-9
    # classes with no launches are left out
    kt[1] = (0.0, 0)
    assert "k_cg_update" not in bench.roofline_of(kt, n, 1, 2098.0, 6791.0, "measured")["classes"]
