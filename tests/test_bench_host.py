"""Host-side logic of bench.py (no GPU): multi-rank aggregation over gloo, and
the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    m = bench.reduce_max(ms, dist, "cpu")
    rate = bench.whole_job_rate(1000, world, m)
    out.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_multirank_takes_the_slowest_rank_and_counts_all_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 15.0                      # max over ranks
        assert abs(rate - 2 * 1000 / 0.015) < 1e-6  # all ranks' cells / slowest time


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--n", "64", "--cpu-sample-n", "16"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "cells/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_traffic_hash_follows_only_the_kernels_own_sources():
    # roofline.traffic is dropped once the counted kernel's sources change: a
    # change to the scan's translation unit leaves the sort's hash alone, a
    # change to a shared header moves every hash
    sys.path.insert(0, ROOT)
    import bench
    d = os.path.join(ROOT, "paper_2109_10375_gb300", "csrc")
    plain = lambda f: open(os.path.join(d, f), "rb").read()
    edit = lambda name: (lambda f: plain(f) + (b"//" if f == name else b""))
    assert bench._src_hash("sort_pass", edit("assign.cu")) == bench._src_hash("sort_pass", plain)
    assert bench._src_hash("scan_assign", edit("assign.cu")) != bench._src_hash("scan_assign", plain)
    assert bench._src_hash("fft_z_conv", edit("sort.cu")) == bench._src_hash("fft_z_conv", plain)
    for k in ("sort_pass", "scan_assign", "fft_r2c_x", "scatter_back"):
        assert bench._src_hash(k, edit("common.cuh")) != bench._src_hash(k, plain)
    t = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    for k, v in t["kernels"].items():
        assert v["src_hash"] and v["bytes_per_launch"] > 0 and v["cells"] > 0, k


def test_model_bytes_follow_the_scope_table():
    # model A: five FFT passes x 8, histogram 4, digit passes 12 + 16 + .. + 12,
    # matching 12 B/cell -- 112 B/cell with four 8-bit passes, 96 with three
    import bench
    for passes, total in ((4, 112), (3, 96)):
        mb = bench.model_bytes(64, passes)
        assert sum(mb.values()) == total * 64 ** 3
        assert mb["sort_pass"] == (total - 56) * 64 ** 3
