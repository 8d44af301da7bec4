"""Permutation classes shared by host and GPU tests (test helper)."""

from oracle import f2
import workloads as wl


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def classes_for(n, e, seed):
    """bit-reversal, half-swap, BP, BPC, tiled-only and dense BMMCs on n bits."""
    k = min(8 - {4: 2, 8: 3, 16: 4}[e], n)
    out = [("bit_reverse", wl.bit_reverse(n), 0),
           ("half_swap", wl.half_swap(n), 0),
           ("bp", wl.random_bp(n, seed), 0),
           ("bpc", wl.random_bp(n, seed + 1), wl.random_c(n, seed))]
    rows, c = wl.tiled_only_bmmc(n, k, seed, _inv)
    out.append(("tiled_only", rows, c))
    rows, c = wl.dense_bmmc(n, seed, _inv)
    out.append(("dense", rows, c))
    return out
