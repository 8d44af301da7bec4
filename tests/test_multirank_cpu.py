"""The N > 1 host logic of bench.py on CPU: two gloo ranks (replicas).

Each rank draws its own workload (seeded by rank), the timing is the max over
ranks and the bytes are the sum, and no collective touches the data path."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        items = bench.workload(12, [4], 2, 1, 2, seed_base=1000 * rank)
        t = bench.allreduce_max(world, 10.0 + rank)
        b = bench.allreduce_sum(world, 100.0 * (rank + 1))
        bench.barrier(world)
        q.put((rank, t, b, [rows for (_, _, rows, _) in items]))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    assert [r[1] for r in results] == [11.0, 11.0]      # max over ranks
    assert [r[2] for r in results] == [300.0, 300.0]    # sum over ranks
    # replicas draw different random matrices (bit-reversal/half-swap agree)
    rows0, rows1 = results[0][3], results[1][3]
    assert rows0[:2] == rows1[:2]
    assert rows0[2:] != rows1[2:]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the other
    ranks exit at once with status 0."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "0"])
    args = bench.parse_args()
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_reports_our_config(monkeypatch, capsys):
    """The reference arm times the oracle on the same workload config as our
    arm's line (here on a small sample size, to keep the test short)."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "ORACLE_N", 12)
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2",
                                      "--warmup", "1"])
    args = bench.parse_args()
    assert bench.reference_arm(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config(args, 1)
    assert line["cpu_baseline"]["value"] == line["value"] > 0
    assert "n = 12" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
