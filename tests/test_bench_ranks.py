"""The multi-rank bench path on the CPU (gloo, world size 2): every rank builds its own seeded
instance (no exchange on the data path), the job time is the slowest rank's, and the job
throughput counts the points of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        e2e = bench.max_over_ranks(0.5 - 0.25 * rank, world, "cpu")
        seed = bench.rank_data_seed(synth.WORKLOADS[bench.WORKLOAD], rank)
        X = synth.mixture(64, 8, synth.U8, 4, 10.0, seed)
        q.put((rank, ms, e2e, bench.job_throughput(1000, world, ms / 1e3), seed, X.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_points():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # the slower rank's step time on every rank
    assert [o[2] for o in out] == [0.5, 0.5]
    assert out[0][3] == pytest.approx(2 * 1000 / 0.015)  # both ranks' points over that time
    assert out[0][4] != out[1][4] and out[0][5] != out[1][5]  # independent instances per rank


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(10, 1, 0.5) == 20.0
