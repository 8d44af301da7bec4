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


def _shard_main(rank, world, port, n, cases, q):
    """One rank of a sharded BMMC over gloo: local steps through the oracle's
    C loop (a CPU stand-in for the kernels), exchanges through gloo's
    all_to_all_single; the result shards are gathered on rank 0."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2306_07795_gb300.shard import ShardedPlan
        import workloads as wl
        g = world.bit_length() - 1
        nl = n - g
        out = []
        for rows, c, e in cases:
            full = wl.payload(n, e, seed=7)
            flat = np.ascontiguousarray(full).reshape(-1).view(np.int32)
            per = flat.size >> g
            mine = torch.from_numpy(flat[rank * per:(rank + 1) * per].copy())

            def local(lrows, lc, x):
                arr = np.ascontiguousarray(x.numpy()).reshape(-1)
                y = oracle.apply(nl, lrows, lc, arr, elem_bytes=e)
                return torch.from_numpy(y).view(x.shape)

            res = ShardedPlan(n, g, rows, c, elem_bytes=e)(mine, rank, local=local)
            parts = [torch.empty_like(res) for _ in range(world)]
            dist.all_gather(parts, res)
            if rank == 0:
                got = torch.cat(parts).numpy()
                want = oracle.apply(n, rows, c, full, elem_bytes=e)
                want = np.ascontiguousarray(want).reshape(-1).view(np.int32)
                out.append(bool(np.array_equal(got, want)))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_bmmc_gloo(world):
    """A BMMC of one array spread over 2 and 4 gloo ranks equals the oracle
    on the whole array, bit for bit (dense matrices with one and two
    exchanges, bit-reversal, 4- and 16-byte elements)."""
    from oracle import f2
    import workloads as wl
    n = 12
    inv = lambda rows: f2.is_invertible(rows, n)  # noqa: E731
    cases = [wl.dense_bmmc(n, 1, inv) + (4,), wl.dense_bmmc(n, 2, inv) + (16,),
             (wl.bit_reverse(n), 0, 4)]
    g = world.bit_length() - 1
    low = (1 << (n - g)) - 1
    # whole shards change rank: no low bit reaches the rank bits (two exchanges)
    lr, lc = wl.dense_bmmc(n - g, 3, lambda r: f2.is_invertible(r, n - g))
    top = [1 << (n - 1 - i) for i in range(g)]
    cases.append((list(lr) + top, (lc & low) | (1 << (n - g)), 8))
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, n, cases, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0] == [True] * len(cases)
