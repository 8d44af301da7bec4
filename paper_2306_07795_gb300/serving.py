"""Request serving: continuous admission of BMMC permutation requests.

Requests arrive over time (each: n, element size, matrix A, complement c,
input array already on the device).  The server

* admits a request as soon as it has arrived, a stream slot is free and its
  device bytes (input + output + workspace) fit in the HBM budget;
* keeps plans in a cache keyed by (n, e, A, c) and output/workspace buffers
  in a pool keyed by size, so steady-state admission allocates nothing new;
* runs admitted requests on S streams, so requests that arrive while others
  are on the GPU start at once and overlap with them on the device; small
  requests admitted in the same scheduling round share one persistent batch
  launch when there are several;
* retires requests as their completion events fire, returning bytes and
  slots, and records each completion time on the GPU clock.

Latency of a request = completion (CUDA event, relative to a start event
recorded when the run begins) - arrival (host clock, relative to the same
instant).  The plain baseline, ``serve_plain``, launches one request at a
time in arrival order on one stream.
"""

import collections
import time

from . import _binding as B
from .plan import Plan


class PlanCache:
    """LRU cache of plans keyed by (n, e, rows, c, flags)."""

    def __init__(self, capacity=4096):
        self.capacity = capacity
        self._d = collections.OrderedDict()
        self.hits = 0
        self.misses = 0

    def get(self, n, rows, c, e, flags):
        key = (n, e, tuple(rows), c, flags)
        p = self._d.get(key)
        if p is not None:
            self._d.move_to_end(key)
            self.hits += 1
            return p
        self.misses += 1
        p = Plan(n, rows, c, e, flags=flags)
        self._d[key] = p
        if len(self._d) > self.capacity:
            self._d.popitem(last=False)
        return p


class BufferPool:
    """Device byte buffers reused by exact size."""

    def __init__(self, device):
        self.device = device
        self._free = collections.defaultdict(list)
        self.allocated_bytes = 0

    def take(self, nbytes):
        import torch
        lst = self._free.get(nbytes)
        if lst:
            return lst.pop()
        self.allocated_bytes += nbytes
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def give(self, buf):
        self._free[buf.numel()].append(buf)


class Request:
    __slots__ = ("rid", "arrival", "n", "e", "rows", "c", "x", "out", "ws",
                 "plan", "done_event", "slot", "bytes", "completion")

    def __init__(self, rid, arrival, n, e, rows, c, x):
        self.rid = rid
        self.arrival = arrival
        self.n = n
        self.e = e
        self.rows = rows
        self.c = c
        self.x = x
        self.out = None
        self.ws = None
        self.plan = None
        self.done_event = None
        self.slot = None
        self.bytes = 0
        self.completion = None


def _percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    k = (len(v) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def summarize(requests, makespan_s):
    lat = [(r.completion - r.arrival) * 1e3 for r in requests]
    moved = sum(2 * (1 << r.n) * r.e for r in requests)
    return {"requests": len(requests),
            "throughput_req_s": len(requests) / makespan_s,
            "effective_gbs": moved / makespan_s / 1e9,
            "p50_ms": _percentile(lat, 0.50), "p99_ms": _percentile(lat, 0.99),
            "mean_ms": sum(lat) / len(lat) if lat else None,
            "makespan_s": makespan_s}


class Server:
    def __init__(self, device, budget_bytes=40 * 10**9, streams=4,
                 flags=B.BMMC_PLAN_PAPER, batch_threshold_bytes=1 << 22,
                 plan_cache=None):
        import torch
        self.device = device
        self.budget = budget_bytes
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.flags = flags
        self.batch_threshold = batch_threshold_bytes
        self.plans = plan_cache or PlanCache()
        self.pool = BufferPool(device)
        self.stats = {"admitted_rounds": 0, "batched_launches": 0, "single_launches": 0,
                      "max_in_flight_bytes": 0, "max_in_flight": 0}

    def _plan(self, r):
        r.plan = self.plans.get(r.n, r.rows, r.c, r.e, self.flags)
        r.bytes = 2 * (1 << r.n) * r.e + r.plan.workspace_bytes  # in + out + ws

    def _buffers(self, r):
        r.out = self.pool.take((1 << r.n) * r.e)
        wsb = r.plan.workspace_bytes
        r.ws = self.pool.take(wsb) if wsb else None

    def _release(self, r, keep_outputs):
        if not keep_outputs:
            self.pool.give(r.out)
        if r.ws is not None:
            self.pool.give(r.ws)
        r.ws = None

    def _launch_single(self, r, stream):
        import torch
        r.plan(r.x, out=_view_like(r.out, r.x), stream=stream,
               workspace=r.ws if r.ws is not None else None)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        r.done_event = ev
        self.stats["single_launches"] += 1

    def _launch_group(self, group, stream):
        import torch
        from .batch import Batch
        b = Batch([r.plan for r in group], [r.x for r in group],
                  [_view_like(r.out, r.x) for r in group],
                  workspace=None, stream=stream)
        b(stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        for r in group:
            r.done_event = ev
        self.stats["batched_launches"] += 1
        return b

    def run(self, requests, poll_s=20e-6, keep_outputs=False):
        """Serve `requests` (sorted by arrival, seconds from start).  Returns
        (finished requests with completion times, makespan in seconds).
        With keep_outputs the output buffers stay with the requests instead of
        returning to the pool."""
        import torch
        torch.cuda.synchronize(self.device)
        start_ev = torch.cuda.Event(enable_timing=True)
        start_ev.record(torch.cuda.current_stream(self.device))
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        pending = collections.deque(requests)
        waiting = collections.deque()  # arrived, not admitted
        # per stream, launches in issue order: (requests, event, batch or None);
        # a stream completes its launches in order, so only heads are polled
        queues = [collections.deque() for _ in self.streams]
        used_bytes = 0
        finished = []
        while pending or waiting or any(queues):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # retire
            for q in queues:
                while q and q[0][1].query():
                    group, _, _ = q.popleft()
                    for r in group:
                        used_bytes -= r.bytes
                        self._release(r, keep_outputs)
                        finished.append(r)
            # admit, in arrival order, while bytes and slots allow
            admitted = []
            while waiting:
                r = waiting[0]
                if r.plan is None:
                    self._plan(r)
                if used_bytes + r.bytes > self.budget and (used_bytes or admitted):
                    break
                waiting.popleft()
                self._buffers(r)
                used_bytes += r.bytes
                admitted.append(r)
            if admitted:
                self.stats["admitted_rounds"] += 1
                small = [r for r in admitted if (1 << r.n) * r.e <= self.batch_threshold]
                large = [r for r in admitted if (1 << r.n) * r.e > self.batch_threshold]
                work = [[r] for r in large]
                if len(small) >= 2:
                    work.append(small)
                else:
                    work.extend([r] for r in small)
                for group in work:
                    si = min(range(len(self.streams)), key=lambda i: len(queues[i]))
                    stream = self.streams[si]
                    keep = None
                    if len(group) == 1:
                        self._launch_single(group[0], stream)
                    else:
                        keep = self._launch_group(group, stream)
                    queues[si].append((group, group[0].done_event, keep))
                self.stats["max_in_flight_bytes"] = max(self.stats["max_in_flight_bytes"],
                                                        used_bytes)
                self.stats["max_in_flight"] = max(
                    self.stats["max_in_flight"],
                    sum(len(g) for q in queues for g, _, _ in q))
            elif not any(queues) and not waiting and pending:
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
            else:
                time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        for r in finished:
            r.completion = start_ev.elapsed_time(r.done_event) / 1e3
        makespan = max(r.completion for r in finished)
        return finished, makespan


def serve_plain(requests, device, flags=B.BMMC_PLAN_PAPER, plan_cache=None,
                keep_outputs=False):
    """Baseline: in arrival order, one plan and one launch per request on a
    single stream, no admission control, no batching.  Buffers of finished
    requests are recycled unless keep_outputs."""
    import torch
    plans = plan_cache or PlanCache()
    stream = torch.cuda.Stream(device=device)
    pool = BufferPool(device)
    torch.cuda.synchronize(device)
    start_ev = torch.cuda.Event(enable_timing=True)
    start_ev.record(torch.cuda.current_stream(device))
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    outs = []
    live = collections.deque()
    for r in requests:
        wait = r.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        while live and live[0].done_event.query():
            done = live.popleft()
            if not keep_outputs:
                pool.give(done.out)
            if done.ws is not None:
                pool.give(done.ws)
            done.ws = None
        r.plan = plans.get(r.n, r.rows, r.c, r.e, flags)
        nb = (1 << r.n) * r.e
        r.out = pool.take(nb)
        wsb = r.plan.workspace_bytes
        r.ws = pool.take(wsb) if wsb else None
        r.plan(r.x, out=_view_like(r.out, r.x), stream=stream, workspace=r.ws)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        r.done_event = ev
        outs.append(r)
        live.append(r)
    torch.cuda.synchronize(device)
    for r in outs:
        r.completion = start_ev.elapsed_time(r.done_event) / 1e3
    makespan = max(r.completion for r in outs)
    return outs, makespan


def _view_like(buf, like):
    return buf.view(like.dtype).view(like.shape)
