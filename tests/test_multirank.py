"""The multi-rank path of the benchmark on the host (gloo, two ranks).

Every rank scores its own dataset; the job's time is the maximum over ranks
and its value counts all ranks' families.  The reference arm under torchrun
runs on rank 0 only and prints one line.
"""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    try:
        bench = _bench()
        total, value = bench._aggregate(10.0 + rank, 1000, 2, 2, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump([total, value], f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank_and_counts_all(tmp_path):
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    for rank in range(2):
        total, value = json.load(open(tmp_path / f"r{rank}.json"))
        assert total == 11.0
        assert value == pytest.approx(2 * 1000 * 2 / 0.011)


def test_single_rank_aggregate_is_the_local_total():
    total, value = _bench()._aggregate(5.0, 100, 4, 1, "cpu")
    assert total == 5.0 and value == pytest.approx(100 * 4 / 0.005)


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def _shard_rank_main(rank, port, out_dir, m, q):
    """Each rank takes its shard of one m-variable table and lists the slots it writes
    (families (c, S) whose sub-walk CTA (S & (2^k-1)) >> W is in the shard's range); the
    ranks exchange the lists and check that they are disjoint and cover the table."""
    import numpy as np
    from paper_1901_07643_gb300 import binding
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    try:
        k, W, b, e = binding.shard_range(1000, m, (rank, 2), q=q)
        half = 1 << (m - 1)
        idx = np.arange(m * half, dtype=np.int64)
        c = idx // half
        comp = idx % half
        S = (comp & ((1 << c) - 1)) | ((comp >> c) << (c + 1))
        g = (S & ((1 << k) - 1)) >> W
        mine = torch.from_numpy(((g >= b) & (g < e)).astype(np.uint8))
        both = [torch.zeros_like(mine) for _ in range(2)]
        dist.all_gather(both, mine)
        total = both[0].int() + both[1].int()
        with open(os.path.join(out_dir, f"s{rank}.json"), "w") as f:
            json.dump([int(total.min()), int(total.max()), int(mine.sum())], f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("m,q", [(16, 6), (13, 7)])
def test_two_rank_shards_cover_the_table_once(tmp_path, m, q):
    mp.start_processes(_shard_rank_main, args=(_free_port(), str(tmp_path), m, q), nprocs=2,
                       start_method="spawn")
    counts = []
    for rank in range(2):
        lo, hi, cnt = json.load(open(tmp_path / f"s{rank}.json"))
        assert lo == 1 and hi == 1
        counts.append(cnt)
    assert sum(counts) == m << (m - 1)  # (13, 7) has one CTA pair: shard 0 is empty
