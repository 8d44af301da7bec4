"""Request serving over the native server of include/bmmc_server.h.

Server(mode="continuous") admits requests as they arrive under an HBM budget
onto S streams (small ones grouped into batch launches); Server(mode="plain")
is the one-launch-per-request baseline.  Both plan in the submitting thread,
inside the library, and time completions with CUDA events; see the header for
the scheduling rules.

drive(server, requests) submits each request at its arrival time (seconds
from the start of the run) and returns per-request latencies.

The paper has no serving counterpart (Sec. 6 times one array at a time);
every request runs the same passes as a plain execution.
"""

import time

from . import _binding as B


class Request:
    """One permutation request: an array of 2^n elements of e bytes already
    on the device (x), a matrix (rows) and complement c, arriving at
    `arrival` seconds."""

    __slots__ = ("rid", "arrival", "n", "e", "rows", "c", "x", "status",
                 "submit_ms", "done_ms", "out_ptr", "late_ms", "arrival_ms", "rows_c")

    def __init__(self, rid, arrival, n, e, rows, c, x):
        self.rid = rid
        self.arrival = arrival
        self.n = n
        self.e = e
        self.rows = rows
        self.c = c
        self.x = x
        self.status = None
        self.submit_ms = None
        self.done_ms = None
        self.out_ptr = None
        self.late_ms = None
        self.arrival_ms = None
        self.rows_c = B.rows_array(rows)  # converted once, outside the timed loop

    @property
    def latency_ms(self):
        """Completion minus scheduled arrival (server clock), so a submitter
        that falls behind does not hide queueing."""
        return self.done_ms - self.arrival_ms


class Server:
    def __init__(self, device, mode="continuous", streams=4, budget_bytes=40 * 10**9,
                 arena_bytes=None, flags=B.BMMC_PLAN_PAPER, group_max_bytes=1 << 22,
                 group_min=4, keep_outputs=False, plan_cache=None, large_log2=None):
        import torch
        self.device = torch.device(device)
        cfg = B.bmmc_server_config()
        cfg.mode = B.BMMC_SERVER_PLAIN if mode == "plain" else B.BMMC_SERVER_CONTINUOUS
        cfg.streams = streams
        cfg.budget_bytes = int(budget_bytes)
        cfg.arena_bytes = int(arena_bytes if arena_bytes is not None else budget_bytes)
        cfg.plan_flags = flags
        cfg.group_max_bytes = int(group_max_bytes)
        cfg.group_min = group_min
        cfg.keep_outputs = 1 if keep_outputs else 0
        # the plain baseline plans every request; the server keeps plans
        if plan_cache is None:
            plan_cache = 0 if mode == "plain" else 1024
        cfg.plan_cache = int(plan_cache)
        # Requests of at least 2^large_log2 bytes (default 256 MiB arrays,
        # whose two passes keep the GPU busy for about 0.16 ms or more) that
        # find the server nearly idle run on a high-priority stream, so that
        # small requests arriving meanwhile take only the SMs they leave idle.
        # 0 = every stream alike.
        if large_log2 is None:
            large_log2 = 28 if mode != "plain" else 0
        cfg.large_log2 = int(large_log2)
        self.mode = mode
        with torch.cuda.device(self.device):
            self._h = B.bmmc_server_create(cfg)

    def submit(self, rid, n, rows, c, elem_bytes, x):
        """Queue one request (x: contiguous CUDA tensor of 2^n * elem_bytes
        bytes).  Returns the library status code."""
        return B.bmmc_server_submit(self._h, rid, n, rows, c, elem_bytes, x.data_ptr())

    def drain(self):
        B.bmmc_server_drain(self._h)

    def hold(self, on=True):
        """Stop (on) or resume admission; queued requests are admitted together
        on resume."""
        B.bmmc_server_hold(self._h, on)

    def now_ms(self):
        return B.bmmc_server_now_ms(self._h)

    def results(self):
        return B.bmmc_server_results(self._h)

    def release(self, ptr):
        B.bmmc_server_release(self._h, ptr)

    def stats(self):
        return B.bmmc_server_stats(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            B.bmmc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def drive(server, requests, spin_s=200e-6):
    """Submit `requests` (sorted by arrival) at their arrival times, wait for
    all of them, and fill in status, submit/done times and outputs.  Returns
    the requests."""
    import torch
    with torch.cuda.device(server.device):
        origin_ms = server.now_ms()  # driver time 0 on the server's clock
        t_start = time.perf_counter()
        by_id = {}
        for r in requests:
            while True:
                wait = r.arrival - (time.perf_counter() - t_start)
                if wait <= 0:
                    break
                if wait > spin_s:
                    time.sleep(wait - spin_s)
            r.late_ms = ((time.perf_counter() - t_start) - r.arrival) * 1e3
            r.arrival_ms = origin_ms + r.arrival * 1e3
            r.status = server.submit(r.rid, r.n, r.rows_c, r.c, r.e, r.x)
            by_id[r.rid] = r
        server.drain()
        for rid, status, sub, done, out in server.results():
            r = by_id[rid]
            r.status = status
            r.submit_ms = sub
            r.done_ms = done
            r.out_ptr = out
    return requests


def _percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    k = (len(v) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def summarize(requests):
    ok = [r for r in requests if r.status == B.BMMC_OK and r.done_ms is not None]
    lat = [r.latency_ms for r in ok]
    first = min(r.arrival_ms for r in ok)
    last = max(r.done_ms for r in ok)
    span_s = (last - first) / 1e3
    moved = sum(2 * (1 << r.n) * r.e for r in ok)
    late = [r.late_ms for r in requests if r.late_ms is not None]
    return {"requests": len(requests), "completed": len(ok),
            "throughput_req_s": len(ok) / span_s, "effective_gbs": moved / span_s / 1e9,
            "p50_ms": _percentile(lat, 0.50), "p99_ms": _percentile(lat, 0.99),
            "mean_ms": sum(lat) / len(lat), "makespan_s": span_s,
            "submit_late_p99_ms": _percentile(late, 0.99)}
