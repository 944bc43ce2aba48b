"""Sharding the batched workload across ranks: the size-balanced assignment and
the gather of per-problem results, on the CPU with two gloo ranks.  Each rank
runs the oracle's adaptive ID on its share of small kernel blocks; rank 0's
gathered results must equal a single-process run of every problem, each
problem run exactly once."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_09417_gb300 import shard  # noqa: E402
from paper_2310_09417_gb300 import workloads as W  # noqa: E402


def test_assign_balances_and_covers():
    rng = np.random.default_rng(1)
    sizes = rng.integers(64, 1025, size=(500, 2))
    costs = [shard.problem_cost(int(m), int(n), int(min(m, n)), 32) for m, n in sizes]
    for world in (1, 2, 3, 8):
        parts = shard.assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        # LPT: the largest load exceeds the mean by at most the largest single cost
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - sum(loads) / world <= max(costs) + 1e-6
        assert shard.imbalance(costs, parts) < 1.02 or world == 1
    assert shard.assign(costs, 4) == shard.assign(costs, 4)  # deterministic
    assert shard.assign([5.0, 5.0, 5.0], 2) == [[0, 2], [1]]


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problems():
    pts, leaves, pairs = W.kernel_block_pairs(6000, 24, 5, leaf_max=128, size_min=32)
    return pts, leaves, pairs


def _run_one(orc, pts, leaves, pair, b=16, tol=1e-8):
    A = W.gaussian_kernel_block(pts, leaves[pair[0]], leaves[pair[1]], h=0.3)
    m, n = A.shape
    Om = orc.gaussian_rows(7, 0, orc.rows_needed(n, b, m=m), m)
    r = orc.id_adaptive(A, Om, b, tol * orc.fro_norm(A))
    return {"k": int(r["k"]), "J": [int(j) for j in r["J"]]}


def _rank(rank, world, port, outdir):
    import torch.distributed as dist

    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts, leaves, pairs = _problems()
        costs = [shard.problem_cost(len(leaves[a]), len(leaves[c]), min(len(leaves[a]), len(leaves[c])), 16)
                 for a, c in pairs]
        mine = shard.assign(costs, world)[rank]
        local = {i: _run_one(orc, pts, leaves, pairs[i]) for i in mine}
        merged = shard.gather_results(local, world, rank)
        if rank == 0:
            with open(os.path.join(outdir, "merged.json"), "w") as f:
                json.dump({str(i): v for i, v in merged.items()}, f)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_batch_equals_single_process(tmp_path, orc):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    merged = {int(i): v for i, v in json.load(open(tmp_path / "merged.json")).items()}
    pts, leaves, pairs = _problems()
    assert sorted(merged) == list(range(len(pairs)))
    for i, pr in enumerate(pairs):
        assert merged[i] == _run_one(orc, pts, leaves, pr)
