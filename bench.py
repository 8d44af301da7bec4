#!/usr/bin/env python3
"""Benchmark of BMMC permutations on GB300: effective bandwidth 2*N*e / time.

Default workload (one "step"): arrays of 2^28 elements at 4, 8 and 16 bytes
per element, and for each element size the permutation set
    bit reversal, half swap (2^14 x 2^14 transpose), 16 random bit
    permutations, 16 random tiled-only BMMCs, 64 random dense BMMCs
(dense BMMCs with a random complement c).  Each permutation runs once per
step through the library's C ABI on device-resident buffers; every array is
larger than L2, so no flush is needed between steps.

Reported beside the headline number: per-class bandwidth, a same-run
cudaMemcpyAsync device-to-device copy of the same bytes, the dominant
kernel's roofline against the measured HBM peak, the end-to-end figure with
host buffers, the SM clocks sampled during the timed region, and the CPU
oracle timed on a bounded sample (baseline only).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 the script runs under torchrun, one process per GPU, each GPU
running the full per-GPU workload (independent arrays: replicas, weak
scaling); the value is the total bytes of all ranks over the slowest rank.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("effective GB/s (2·N·bytes/s) vs GB300 HBM peak & D2D copy; "
          "batched/served p50/p99")
FALLBACK_HBM_GBS = 6800.0
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "bmmc_tiled_pass_traffic.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2306_07795_gb300", "csrc", f)
                  for f in ("kernels.cu", "pass_desc.h", "plan.cpp")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--elem", type=str, default="4,8,16")
    ap.add_argument("--dense", type=int, default=64)
    ap.add_argument("--bp", type=int, default=16)
    ap.add_argument("--tiled", type=int, default=16)
    ap.add_argument("--strategy", choices=["paper", "single"], default="paper")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# Distributed setup (replicas; no collective on the data path)
# ---------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# Workload
# ---------------------------------------------------------------------------

def lib_invertible(n):
    """Invertibility test for rejection sampling: the library's own
    validation (bmmc_plan_create returns BMMC_ERR_SINGULAR)."""
    import paper_2306_07795_gb300 as bm

    def test(rows):
        try:
            h = bm.bmmc_plan_create(n, rows, 0, 4)
        except bm.BmmcError as err:
            if err.code == bm.BMMC_ERR_SINGULAR:
                return False
            raise
        bm.bmmc_plan_destroy(h)
        return True
    return test


def workload(n, elems, n_bp, n_tiled, n_dense, seed_base=0):
    """List of (class, e, rows, c) for one step."""
    import workloads as wl
    inv = lib_invertible(n)
    out = []
    for e in elems:
        k = 8 - {4: 2, 8: 3, 16: 4}[e]
        out.append(("bit_reverse", e, wl.bit_reverse(n), 0))
        out.append(("half_swap", e, wl.half_swap(n), 0))
        for s in range(n_bp):
            out.append(("bp", e, wl.random_bp(n, seed_base + 1 + s), 0))
        for s in range(n_tiled):
            rows, c = wl.tiled_only_bmmc(n, k, seed_base + 1 + s, inv)
            out.append(("tiled_only", e, rows, c))
        for s in range(n_dense):
            rows, c = wl.dense_bmmc(n, seed_base + 1 + s, inv)
            out.append(("dense", e, rows, c))
    return out


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,"
               "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap")


def clock_sampler_start(device_index):
    import torch
    sel = []
    try:
        uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        if uuid:
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
    except Exception:
        sel = []
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=" + CLOCK_QUERY,
             "--format=csv,noheader,nounits", "-lms", "200"] + sel,
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except (OSError, FileNotFoundError):
        return None


def clock_sampler_stop(proc):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    time.sleep(0.25)
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, power = [], [], []
    flags = {"hw_slowdown": 0, "hw_thermal_slowdown": 0,
             "sw_thermal_slowdown": 0, "sw_power_cap": 0}
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
             "sw_power_cap"]
    for line in out.splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
            power.append(float(parts[3]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                flags[nm] += 1
    reasons = [nm for nm in names if flags[nm]]
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm), "reasons": reasons}


# ---------------------------------------------------------------------------
# Roofline helpers
# ---------------------------------------------------------------------------

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            peaks = json.load(f)
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources for this kernel; else None."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            text = f.read()
    except OSError:
        return None, None
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            key, val = line[2:].split(":", 1)
            fields[key.strip()] = val.strip().strip("`")
    if fields.get("source_sha") != kernel_source_sha():
        return None, "stale"
    if fields.get("kernel") != kernel_name:
        return None, "other kernel"
    try:
        return float(fields["dram_bytes_per_launch"]), fields.get("workload")
    except (KeyError, ValueError):
        return None, None


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(n_sample=24, elems=(4, 8, 16)):
    """One permutation of each class per element size, at 2^n_sample
    elements: a bounded sample of the benchmark workload."""
    import workloads as wl
    from oracle import f2
    inv = lambda rows: f2.is_invertible(rows, len(rows))  # noqa: E731
    items = []
    for e in elems:
        k = 8 - {4: 2, 8: 3, 16: 4}[e]
        items.append(("bit_reverse", e, wl.bit_reverse(n_sample), 0))
        items.append(("half_swap", e, wl.half_swap(n_sample), 0))
        items.append(("bp", e, wl.random_bp(n_sample, 1), 0))
        rows, c = wl.tiled_only_bmmc(n_sample, k, 1, inv)
        items.append(("tiled_only", e, rows, c))
        rows, c = wl.dense_bmmc(n_sample, 1, inv)
        items.append(("dense", e, rows, c))
    return items


def run_oracle_step(n_sample, items, buffers):
    import oracle
    moved = 0
    for cls, e, rows, c in items:
        inp = buffers[e]
        oracle.apply(n_sample, rows, c, inp, elem_bytes=e)
        moved += 2 * (1 << n_sample) * e
    return moved


def cpu_baseline(n_sample=24, reps=1):
    import oracle
    import workloads as wl
    items = oracle_sample(n_sample)
    buffers = {e: wl.payload(n_sample, e) for e in (4, 8, 16)}
    run_oracle_step(n_sample, items[:1], buffers)  # warm the library
    t0 = time.perf_counter()
    moved = 0
    for _ in range(reps):
        moved += run_oracle_step(n_sample, items, buffers)
    dt = time.perf_counter() - t0
    return {"value": moved / dt / 1e9, "unit": "GB/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": ("C loop out[A x + c] = in[x] (OpenMP over x), 2^%d elements, "
                       "one bit-reversal, half-swap, random BP, tiled-only and dense "
                       "BMMC at each of 4, 8, 16 bytes per element; %d pass(es), "
                       "%.1f s" % (n_sample, reps, dt))}


def reference_arm(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    import oracle
    import workloads as wl
    n_sample = 24
    items = oracle_sample(n_sample)
    buffers = {e: wl.payload(n_sample, e) for e in (4, 8, 16)}
    for _ in range(args.warmup):
        run_oracle_step(n_sample, items, buffers)
    t0 = time.perf_counter()
    moved = 0
    for _ in range(args.steps):
        moved += run_oracle_step(n_sample, items, buffers)
    dt = time.perf_counter() - t0
    value = moved / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "n=28 BMMC permutation set (bounded 2^24 sample)",
                   "n": n_sample, "elem_bytes": [4, 8, 16]},
        "cpu_baseline": {"value": value, "unit": "GB/s",
                         "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "2^24 elements, one permutation of each class "
                                   "per element size, per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import paper_2306_07795_gb300 as bm

    world, rank, local = dist_setup()
    dist_init(world, local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    elems = [int(v) for v in args.elem.split(",")]
    n = args.n
    N = 1 << n
    flags = bm.BMMC_PLAN_SINGLE_PASS if args.strategy == "single" else bm.BMMC_PLAN_PAPER

    # ---- plans and device buffers (outside the timed region) --------------
    import workloads as wl
    items = workload(n, elems, args.bp, args.tiled, args.dense, seed_base=1000 * rank)
    plans = [bm.Plan(n, rows, c, e, flags=flags) for (_, e, rows, c) in items]
    bufs = {}
    for e in elems:
        x = wl.payload_torch(n, e, seed=rank, device=dev)
        y = torch.empty_like(x)
        ws = torch.empty(N * e, dtype=torch.uint8, device=dev)
        bufs[e] = (x, y, ws)
    torch.cuda.synchronize(dev)

    def run(i):
        cls, e, rows, c = items[i]
        x, y, ws = bufs[e]
        plans[i](x, out=y, stream=stream, workspace=ws)

    # ---- timed region ------------------------------------------------------
    K, W = args.steps, args.warmup
    for _ in range(W):
        for i in range(len(items)):
            run(i)
    per_item = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                for _ in range(len(items) * K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    barrier(world)
    sampler = clock_sampler_start(local)
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    t_start.record(stream)
    for k in range(K):
        for i in range(len(items)):
            ev = per_item[k * len(items) + i]
            ev[0].record(stream)
            run(i)
            ev[1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    wall1 = time.perf_counter()
    clocks = clock_sampler_stop(sampler)
    barrier(world)
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms = allreduce_max(world, elapsed_ms)

    bytes_per_step = sum(2 * N * e for (_, e, _, _) in items)
    total_bytes = allreduce_sum(world, float(bytes_per_step * K))
    value = total_bytes / (elapsed_ms / 1e3) / 1e9
    launches_per_step = sum(p.num_passes for p in plans)

    # per class / element size; per kernel instantiation (one per elem size)
    durs = [0.0] * len(items)
    for k in range(K):
        for i in range(len(items)):
            ev = per_item[k * len(items) + i]
            durs[i] += ev[0].elapsed_time(ev[1]) / K
    by_class = {}
    kernel_time = {}
    kernel_launches = {}
    kernel_bytes = {}
    for i, (cls, e, rows, c) in enumerate(items):
        key = "%s_e%d" % (cls, e)
        b = 2 * N * e
        d = by_class.setdefault(key, {"bytes": 0, "ms": 0.0, "count": 0,
                                      "passes": plans[i].num_passes})
        d["bytes"] += b
        d["ms"] += durs[i]
        d["count"] += 1
        kname = "bmmc_tiled_pass<%d>" % {4: 2, 8: 3, 16: 4}[e]
        kernel_time[kname] = kernel_time.get(kname, 0.0) + durs[i]
        kernel_launches[kname] = kernel_launches.get(kname, 0) + plans[i].num_passes
        kernel_bytes[kname] = kernel_bytes.get(kname, 0) + b * plans[i].num_passes

    # ---- same-run D2D copy baseline ---------------------------------------
    d2d = {}
    for e in elems:
        x, y, _ = bufs[e]
        for _ in range(3):
            y.copy_(x)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(10)]
        for a, b in evs:
            a.record(stream)
            y.copy_(x)
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        d2d[e] = 2 * N * e / (ms / 1e3) / 1e9
    breakdown = {}
    for key, d in sorted(by_class.items()):
        e = int(key.rsplit("_e", 1)[1])
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
        breakdown[key] = {"gbs": round(gbs, 1), "frac_of_d2d": round(gbs / d2d[e], 4),
                          "passes": d["passes"], "count": d["count"]}

    # ---- roofline of the dominant kernel ----------------------------------
    dom = max(kernel_time, key=kernel_time.get)
    avg_launch_ms = kernel_time[dom] / kernel_launches[dom]
    bytes_per_launch = kernel_bytes[dom] / kernel_launches[dom]
    achieved = bytes_per_launch / (avg_launch_ms / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    traffic, traffic_note = profiled_traffic(dom)
    step_ms_sum = sum(kernel_time.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": round(avg_launch_ms, 4),
                "share_of_step": round(kernel_time[dom] / step_ms_sum, 4)}
    if traffic_note and traffic is None:
        roofline["traffic_note"] = traffic_note

    extras = {}
    # ---- single-pass strategy on the dense set (beyond the paper) ---------
    if not args.no_extras and args.strategy == "paper":
        sp = {}
        for e in elems:
            dense = [(rows, c) for (cls, ee, rows, c) in items if cls == "dense" and ee == e]
            if not dense:
                continue
            sp_plans = [bm.Plan(n, rows, c, e, flags=bm.BMMC_PLAN_SINGLE_PASS)
                        for rows, c in dense[:16]]
            x, y, ws = bufs[e]
            for p in sp_plans:
                p(x, out=y, stream=stream)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            for _ in range(2):
                for p in sp_plans:
                    p(x, out=y, stream=stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            gbs = 2 * len(sp_plans) * 2 * N * e / (a.elapsed_time(b) / 1e3) / 1e9
            sp["dense_e%d" % e] = {"gbs": round(gbs, 1), "frac_of_d2d": round(gbs / d2d[e], 4),
                                   "passes": 1, "count": len(sp_plans)}
        extras["single_pass_dense"] = sp

    # ---- end to end through the public API with host buffers --------------
    e2e = None
    if not args.no_e2e:
        host = {}
        for e in elems:
            x, y, _ = bufs[e]
            hin = torch.empty(x.numel(), dtype=x.dtype, pin_memory=True)
            hin.copy_(x)
            hout = torch.empty_like(hin, pin_memory=True)
            host[e] = (hin, hout)
        torch.cuda.synchronize(dev)

        def e2e_step():
            for i, (cls, e, rows, c) in enumerate(items):
                x, y, ws = bufs[e]
                hin, hout = host[e]
                x.copy_(hin, non_blocking=True)
                plans[i](x, out=y, stream=stream, workspace=ws)
                hout.copy_(y, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize(dev)
        barrier(world)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = allreduce_max(world, a.elapsed_time(b))
        e2e_bytes = allreduce_sum(world, float(bytes_per_step * args.e2e_steps))
        hbytes = sum(N * e for (_, e, _, _) in items)
        e2e = {"value": round(e2e_bytes / (ms / 1e3) / 1e9, 1), "unit": "GB/s",
               "h2d_bytes_per_step": hbytes, "d2h_bytes_per_step": hbytes,
               "steps": args.e2e_steps, "warmup": 1}
        del host

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(reps=20)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s",
            "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(elapsed_ms / K, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {
                "workload": "n=28 BMMC permutation set per elem size: bit-reversal, "
                            "half-swap, %d random BP, %d random tiled-only, %d random "
                            "dense (random c)" % (args.bp, args.tiled, args.dense),
                "n": n, "elem_bytes": elems, "strategy": args.strategy,
                "permutations_per_step": len(items),
                "l2": "inputs larger than L2 (%d-%d MiB per array), no flush"
                      % (N * min(elems) >> 20, N * max(elems) >> 20),
                "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * K,
            "clocks": clocks,
            "d2d_copy_gbs": {str(e): round(v, 1) for e, v in d2d.items()},
            "frac_of_d2d": round(value / (sum(d2d[e] * sum(1 for it in items if it[1] == e) * e
                                              for e in elems)
                                          / sum(it[1] for it in items)), 4),
            "breakdown": breakdown,
            "wall_s_timed": round(wall1 - wall0, 3),
        }
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
