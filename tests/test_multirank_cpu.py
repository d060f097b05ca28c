"""World-size-2 tests of the multi-rank host logic on CPU (gloo):
spin sharding + the one signal all-reduce, and bench.py's max-over-ranks
timing and rank-0-only reference arm."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2301_02702_b300.shard import shard_phantom, shard_range
from paper_2301_02702_b300.workloads import random_sequence, random_spins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 100, 262144):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def test_grouped_shards_keep_groups_whole():
    ph = random_spins(50, seed=1)
    ph.group_offsets = np.array([0, 10, 10, 25, 40, 50])
    rows = []
    for r in range(3):
        part, (g_lo, g_hi) = shard_phantom(ph, r, 3)
        rows.append((g_lo, g_hi))
        if g_hi > g_lo:
            assert part.group_offsets[0] == 0 and part.group_offsets[-1] == part.n
    assert rows[0][0] == 0 and rows[-1][1] == 5
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))


def _worker(rank, world, port, grouped, out_q):
    import torch.distributed as dist
    from paper_2301_02702_b300.shard import simulate_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ph = random_spins(37, seed=5)
    if grouped:
        ph.group_offsets = np.array([0, 4, 9, 9, 30, 37])
    seq = random_sequence(120, seed=6)
    sig = simulate_sharded(ph, seq, lambda p, s: oracle.simulate(p, s, threads=1), rank, world)
    import bench
    m = bench.reduce_max(float(rank + 1), world)
    dist.destroy_process_group()
    out_q.put((rank, sig, m))


@pytest.mark.parametrize("grouped", [False, True])
def test_two_rank_sharded_signal_equals_whole(grouped):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, grouped, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ph = random_spins(37, seed=5)
    if grouped:
        ph.group_offsets = np.array([0, 4, 9, 9, 30, 37])
    whole = oracle.simulate(ph, random_sequence(120, seed=6), threads=1)
    for rank, sig, m in res:
        assert m == 2.0  # max over ranks
        assert np.max(np.abs(sig - whole)) <= 1e-12 * np.max(np.abs(whole))


def test_reference_arm_under_torchrun_two_ranks():
    """Rank 0 prints the one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "gre32", "--reference-budget-s", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _failing_worker(rank, world, port, out_q):
    """Rank 1's shard computation fails (a host-side injected fault) and that
    rank exits; rank 0 must learn of it from the collective's error within the
    process group's timeout instead of waiting for ever."""
    import datetime
    import time
    import torch.distributed as dist
    from paper_2301_02702_b300.shard import simulate_sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    ph = random_spins(20, seed=5)
    seq = random_sequence(60, seed=6)

    def shard(p, s):
        if rank == 1:
            raise RuntimeError("injected shard failure")
        return oracle.simulate(p, s, threads=1)

    t0 = time.monotonic()
    try:
        simulate_sharded(ph, seq, shard, rank, world)
        out_q.put((rank, "completed", time.monotonic() - t0))
    except Exception as e:  # noqa: BLE001 - the failure is the point
        out_q.put((rank, f"failed: {type(e).__name__}", time.monotonic() - t0))
        if rank == 1:
            out_q.close()
            out_q.join_thread()  # deliver the report before leaving
            os._exit(3)  # the failed rank leaves without joining the collective
    dist.destroy_process_group()


def test_shard_failure_is_detected_by_the_other_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (status, dt)) for r, status, dt in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
    assert res[1][0].startswith("failed")
    assert res[0][0].startswith("failed"), res  # rank 0's all-reduce reported the lost peer
    assert res[0][1] < 60.0
    assert procs[1].exitcode == 3
