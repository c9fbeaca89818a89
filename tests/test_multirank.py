"""The multi-rank host logic of bench.py on CPU with the gloo backend (world
size 2): the timed region's barrier and max over ranks, the whole-job
throughput, and the reference arm, which runs on rank 0 only.  The apply itself
is per-rank (replicas, no collective on the data path), so nothing else in the
N > 1 path differs from N = 1."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 17.25][rank]            # rank 1 is the slow one
        dist.barrier()
        total = bench.max_over_ranks(local_ms, torch.device("cpu"))
        ms, value = bench.job_throughput(256 ** 3, world, total, 5)
        out.put((rank, total, ms, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, ms, value in res:
        assert total == 17.25                       # the slowest rank's time, on every rank
        assert ms == pytest.approx(17.25 / 5)
        assert value == pytest.approx(2 * 256 ** 3 / (17.25 / 5 / 1e3) / 1e6)


def test_single_process_reduction_is_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    ms, value = bench.job_throughput(100, 1, 50.0, 10)
    assert ms == 5.0 and value == pytest.approx(100 / 5e-3 / 1e6)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_runs_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1", "--ref-n", "16"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    if rank == 1:
        assert lines == []
    else:
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
        assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


# --- sharding a batch of independent applies (LPT) -------------------------------

def _lpt_case(sizes, world):
    import paper_1501_04438_gb300 as gsm
    parts = gsm.partition_batch(sizes, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))                  # every instance exactly once
    return parts, [sum(gsm.apply_cost(sizes[i]) for i in p) for p in parts]


def test_partition_batch_within_graham_bound_of_the_optimum():
    """LPT against the exact optimum (all assignments) on small batches."""
    import itertools
    import paper_1501_04438_gb300 as gsm
    rng = np.random.default_rng(7)
    for trial in range(20):
        world = int(rng.integers(2, 4))
        sizes = [int(v) for v in rng.choice([16, 24, 32, 48, 64], size=int(rng.integers(3, 8)))]
        _, loads = _lpt_case(sizes, world)
        costs = [gsm.apply_cost(n) for n in sizes]
        opt = min(max(sum(c for c, a in zip(costs, assign) if a == r) for r in range(world))
                  for assign in itertools.product(range(world), repeat=len(sizes)))
        assert max(loads) <= (4 / 3 - 1 / (3 * world)) * opt * (1 + 1e-12), (sizes, world)


def test_partition_batch_of_the_uneven_48():
    from paper_1501_04438_gb300 import workloads as wl
    sizes = [n for n, _ in wl.batch_specs()]
    for world in (1, 2, 4, 8):
        parts, loads = _lpt_case(sizes, world)
        assert len(parts) == world
        assert max(loads) / (sum(loads) / world) < 1.05


def _shard_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_1501_04438_gb300 as gsm
    from paper_1501_04438_gb300 import workloads as wl
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sizes = [n for n, _ in wl.batch_specs()]
        mine = gsm.partition_batch(sizes, world)[rank]      # the same on every rank: no exchange needed
        got = [None] * world
        dist.all_gather_object(got, mine)                   # only to check the shards here
        out.put((rank, mine, got))
    finally:
        dist.destroy_process_group()


def test_batch_shards_are_disjoint_and_complete_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, got in res:
        assert got[rank] == mine
        flat = sorted(i for g in got for i in g)
        assert flat == list(range(48))
