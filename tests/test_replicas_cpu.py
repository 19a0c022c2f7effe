"""The multi-GPU form of the bench is replicas only: N independent controllers, the
worst replica's latency and the aggregate frame rate.  The rank logic runs here on
CPU as two gloo ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: latencies 10 + r us, with rank 1 worse in p99 only
    stats = {k: 10.0 + rank for k in bench.REPLICA_STATS}
    stats["p99"] = 30.0 if rank == 1 else 12.0
    stats["mean"] = 20.0 * (rank + 1)
    worst, fps = bench.reduce_replicas(torch, dist, stats, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (worst, fps)


def test_two_gloo_ranks_give_worst_latency_and_summed_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        worst, fps = res[r]
        assert worst["p50"] == 11.0 and worst["p99"] == 30.0 and worst["mean"] == 40.0
        assert fps == pytest.approx(1e6 / 20.0 + 1e6 / 40.0)
    assert res[0] == res[1]


def test_one_rank_needs_no_process_group():
    stats = {k: 5.0 for k in bench.REPLICA_STATS}
    worst, fps = bench.reduce_replicas(torch, None, stats, torch.device("cpu"))
    assert worst == stats and fps == pytest.approx(2e5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.reference(args)
    assert capsys.readouterr().out == ""
