"""Autotuner for the tile options of plans and batches.

The planner fixes the shared-memory swizzle and the lane assignment
analytically (conflict-free layouts are found by a rank search at planning
time).  What it cannot know is how the segment length (seg_bits, the
paper's n_tile) and the bytes per thread block (cta_tile_log2) trade DRAM
locality against occupancy on a given GPU and array size; this module times
candidates on the device and keeps the fastest.

Results for single plans are cached in a JSON file keyed by
(n, element bytes, strategy, passes), so a size class is tuned once.
"""

import json
import os
import statistics

from . import _binding as B
from .plan import Plan

# (seg_bits, cta_tile_log2); 0 = the planner's default
DEFAULT = (0, 0)
CANDIDATES = {
    4: [(0, 0), (5, 13), (5, 14), (6, 13), (6, 15), (7, 15), (7, 16)],
    8: [(0, 0), (4, 13), (4, 14), (5, 13), (5, 15), (6, 15), (6, 16)],
    16: [(0, 0), (3, 13), (3, 14), (4, 13), (4, 15), (5, 15), (5, 16)],
}


def _time_ms(fn, dev, reps):
    import torch
    s = torch.cuda.current_stream(dev)
    fn()
    torch.cuda.synchronize(dev)
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize(dev)
        out.append(a.elapsed_time(b))
    return statistics.median(out)


def tune_batch(make_batch, dev, candidates=None, reps=3):
    """make_batch(seg_bits, cta_tile_log2) -> Batch.  Returns the fastest
    (seg_bits, cta_tile_log2) and the list of trials."""
    trials = []
    for seg, tile in candidates or CANDIDATES[4]:
        try:
            b = make_batch(seg, tile)
        except B.BmmcError:
            continue
        ms = _time_ms(b, dev, reps)
        trials.append({"seg_bits": seg, "cta_tile_log2": tile, "ms": round(ms, 4)})
        del b
    best = min(trials, key=lambda t: t["ms"])
    return (best["seg_bits"], best["cta_tile_log2"]), trials


class TuneCache:
    """JSON-backed cache of tuned plan options."""

    def __init__(self, path=None):
        self.path = path or os.environ.get(
            "BMMC_TUNE_CACHE",
            os.path.join(os.path.expanduser("~"), ".cache", "bmmc_gb300", "tune.json"))
        self.data = {}
        try:
            with open(self.path) as f:
                self.data = json.load(f)
        except (OSError, ValueError):
            self.data = {}

    @staticmethod
    def key(n, e, flags, passes):
        return "%d/%d/%d/%d" % (n, e, flags, passes)

    def get(self, n, e, flags, passes):
        v = self.data.get(self.key(n, e, flags, passes))
        return tuple(v) if v else None

    def put(self, n, e, flags, passes, value):
        self.data[self.key(n, e, flags, passes)] = list(value)
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune_plan(n, rows, c, elem_bytes, dev, flags=B.BMMC_PLAN_PAPER, cache=None,
              reps=5):
    """Fastest (seg_bits, cta_tile_log2) for this permutation's size class,
    timed on device buffers of 2^n elements; cached by size class."""
    import torch
    probe = Plan(n, rows, c, elem_bytes, flags=flags)
    cache = cache if cache is not None else TuneCache()
    hit = cache.get(n, elem_bytes, flags, probe.num_passes)
    if hit is not None:
        return hit
    x = torch.zeros((1 << n) * elem_bytes // 4, dtype=torch.int32, device=dev)
    y = torch.empty_like(x)
    ws = torch.empty(max(probe.workspace_bytes, 16), dtype=torch.uint8, device=dev)
    best, best_ms = DEFAULT, None
    for seg, tile in CANDIDATES[elem_bytes]:
        try:
            p = Plan(n, rows, c, elem_bytes, flags=flags, seg_bits=seg, cta_tile_log2=tile)
        except B.BmmcError:
            continue
        ms = _time_ms(lambda: p(x, out=y, workspace=ws), dev, reps)
        if best_ms is None or ms < best_ms:
            best, best_ms = (seg, tile), ms
    cache.put(n, elem_bytes, flags, probe.num_passes, best)
    return best
