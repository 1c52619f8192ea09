"""Host logic of bench.py's multi-GPU mode (independent replicas, one per rank)
on CPU: two gloo ranks meet at the barriers, both see the slowest rank's time,
and the whole-job rate counts every rank's units over that time."""
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_local, out_q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reps = bench.Replicas(dist, device="cpu")
        assert bench.dist_env() == (world, rank, rank)
        reps.barrier()
        ms = reps.max_over_ranks(ms_local)
        rate = bench.whole_job_rate(world, 1000, ms)
        reps.barrier()
        out_q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times[r], q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, ms, rate in got:
        assert ms == 20.0  # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000 / 0.020)


def test_single_process_replicas_are_identity():
    sys.path.insert(0, ROOT)
    import bench

    reps = bench.Replicas(None)
    reps.barrier()
    assert reps.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 500, 250.0) == pytest.approx(2000.0)


def test_reference_arm_on_other_ranks_does_no_work(monkeypatch, capsys):
    # under torchrun only rank 0 runs the oracle and prints; the others exit quietly
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setitem(sys.modules, "oracle", None)  # importing it would fail: proves it is not reached
    args = bench.argparse.Namespace(steps=1, warmup=0, particles=4096, impl="reference", gpus=2)
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_reference_arm_line(monkeypatch, capsys):
    # rank 0 prints one contract line for the oracle on a small block
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    args = bench.argparse.Namespace(steps=1, warmup=0, particles=4096, impl="reference", gpus=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
