"""bench.py's whole-job figures over several ranks, on the CPU with two gloo ranks.

With N ranks each rank runs its own ID (a replica with its own seed, no
collective on the data path).  The reported step time is the slowest rank's,
and the throughput counts the work of every rank, which may differ when the
replicas stop at different ranks."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402

# per-rank step time (ms) and algorithmic flops of two replicas
MS = [12.5, 20.0]
FLOPS = [3.0e9, 5.5e9]


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.over_ranks(MS[rank], "max", world, "cpu")
        fl = bench.over_ranks(FLOPS[rank], "sum", world, "cpu")
        with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
            json.dump({"ms": ms, "flops": fl}, f)
    finally:
        dist.destroy_process_group()


def test_one_rank_is_the_identity():
    assert bench.over_ranks(7.25, "max", 1, None) == 7.25
    assert bench.over_ranks(7.25, "sum", 1, None) == 7.25


def test_two_gloo_ranks_take_the_slowest_time_and_all_the_work(tmp_path):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for r in range(2):
        got = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert got["ms"] == max(MS)
        assert got["flops"] == sum(FLOPS)
    # the whole-job throughput bench.py reports from them
    value = sum(FLOPS) / (max(MS) * 1e-3) / 1e9
    assert value == pytest.approx(425.0)
