"""bench.py with N > 1 ranks runs independent replicas: the only exchange is the
whole-job aggregation (species-steps summed, time = slowest rank). Tested with two
gloo ranks on the CPU; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.aggregate_over_ranks(1000 * (rank + 1), 0.5 + rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_work_and_take_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: (3000.0, 1.5), 1: (3000.0, 1.5)}


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(123, 4.5) == (123.0, 4.5)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"ref_procs": 1, "species": 1000, "warmup": 3, "steps": 1, "gpus": 2})()
    assert bench.run_reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_shard_trains_covers_every_train_once_and_balances():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    sizes = list(np.geomspace(1e4, 2e6, 64).astype(int))
    for world in (1, 2, 3, 8):
        parts = bench.shard_trains(sizes, world)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(64))
        loads = [sum(sizes[b] for b in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)


def _batched_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        counts = np.zeros((4, 7), dtype=np.int64)
        for b in bench.shard_trains([10, 20, 30, 40], world)[rank]:
            counts[b] = b + 1
        ss, t, c = bench.gather_batched(100 * (rank + 1), 2.0 + rank, counts)
        q.put((rank, ss, t, c.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_sharded_sweep():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ss, t, c in got:
        assert ss == 300.0 and t == 3.0
        assert c == [[b + 1] * 7 for b in range(4)]


def _rows_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the hybrid and volume legs: each train's float row filled on its own rank only
        rows = np.zeros((5, 3))
        for b in bench.shard_trains([50, 10, 40, 20, 30], world)[rank]:
            rows[b] = [b + 0.25, 1.0 / (b + 1), -b]
        q.put((rank, bench.sum_over_ranks(rows).tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_per_train_rows():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rows_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [[b + 0.25, 1.0 / (b + 1), -b] for b in range(5)]
    for rank, rows in got:
        assert rows == want


def test_recorded_traffic_only_while_the_sources_match(tmp_path, monkeypatch):
    import json
    sys.path.insert(0, ROOT)
    import bench
    rec = {"dram_bytes_per_launch": {"k_search_tps": 123, "k_diffuse": 45},
           "sources_sha256": bench.sources_digest(), "tuning": [8, 384, 0, 1]}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.recorded_traffic("k_search_tps") == 123
    assert bench.recorded_traffic("k_sort_pass") is None
    rec["sources_sha256"] = "0" * 64  # the kernels changed since the capture
    path.write_text(json.dumps(rec))
    assert bench.recorded_traffic("k_search_tps") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.recorded_traffic("k_search_tps") is None



def test_sources_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    """The traffic record stays valid across comment and layout edits of the device
    sources and is dropped by any change to the code itself."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2509_03313_gb300", "csrc"), root / "paper_2509_03313_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), root / "include")
    monkeypatch.setattr(bench, "ROOT", str(root))
    base = bench.sources_digest()
    f = root / "paper_2509_03313_gb300" / "csrc" / "phases.cuh"
    text = f.read_text()
    f.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n\n", "\n\n\n", 3))
    assert bench.sources_digest() == base
    f.write_text(text.replace("constexpr int TPS_UNROLL = 4;", "constexpr int TPS_UNROLL = 2;"))
    assert bench.sources_digest() != base
    f.write_text(text)
    (root / "paper_2509_03313_gb300" / "csrc" / "chem_api.cu").write_text("// host code only\n")
    assert bench.sources_digest() == base  # host-only unit left out
