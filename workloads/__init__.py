"""Seeded synthetic inputs shared by the tests, the benchmark and smoke().

This module generates inputs only.  It holds none of the method's arithmetic:
no matrix products, ranks, inverses or index maps.  Where a workload needs an
invertible matrix, the caller supplies the invertibility test (the oracle's in
the tests, the library's own plan validation in the benchmark), and this
module only draws candidates from a seeded stream until one passes.

All randomness comes from numpy's PCG64 generator, which gives the same
stream on x86_64 and aarch64 for the same seed.

Workloads (arrays of 2^n elements of e bytes; matrices as n row masks, bit j
of rows[i] is the entry a_ij):

* bit reversal, y_i = x_{n-1-i}                       (Sec. 1, Sec. 3)
* half swap, p(b) = (b + n/2) mod n: the 2^(n/2) x 2^(n/2) transpose
* random bit permutations (BP, c = 0)                  (Sec. 3, Sec. 6 results)
* random tiled-only BMMCs: k columns S with an invertible k x k block on the
  k low rows, zeros below it, an invertible block on the other rows and
  columns, and random bits elsewhere                   (Sec. 5.1 condition)
* dense random BMMCs: uniform bits, rejection-sampled until invertible, with a
  uniform complement vector c                          (Sec. 6 "random BMMC")
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_bits(g, nbits):
    """A uniform nbits-bit integer (nbits <= 63)."""
    if nbits == 0:
        return 0
    return int(g.integers(0, 1 << nbits, dtype=np.int64))


def _rand_rows(g, n):
    """n uniform n-bit row masks."""
    return [int(v) for v in g.integers(0, 1 << n, size=n, dtype=np.int64)]


# ---------------------------------------------------------------------------
# Matrices
# ---------------------------------------------------------------------------

def bp_rows(p):
    """Row masks of the bit permutation sending input bit b to output bit p[b]."""
    rows = [0] * len(p)
    for b, pb in enumerate(p):
        rows[pb] |= 1 << b
    return rows


def bit_reverse(n):
    return bp_rows([n - 1 - b for b in range(n)])


def half_swap(n):
    """Swap the two halves of the index bits: the transpose of a
    2^(n/2) x 2^(n/2) row-major matrix when n is even."""
    h = n // 2
    return bp_rows([(b + h) % n for b in range(n)])


def identity_rows(n):
    return [1 << b for b in range(n)]


def random_perm(n, seed):
    return [int(v) for v in rng(seed).permutation(n)]


def random_bp(n, seed):
    return bp_rows(random_perm(n, seed))


def random_c(n, seed):
    return _rand_bits(rng(seed ^ 0x5EED_C0DE), n)


def dense_candidates(n, seed):
    """Endless stream of uniform random n x n bit matrices (row masks)."""
    g = rng(seed)
    while True:
        yield _rand_rows(g, n)


def first_passing(candidates, accept):
    """The first candidate for which accept(candidate) is true."""
    for cand in candidates:
        if accept(cand):
            return cand
    raise RuntimeError("unreachable")


def dense_bmmc(n, seed, is_invertible):
    """A uniform random invertible matrix (rejection sampling) and a uniform c.

    ``is_invertible(rows)`` is supplied by the caller.
    """
    rows = first_passing(dense_candidates(n, seed), is_invertible)
    return rows, random_c(n, seed)


def tiled_only_candidates(n, k, seed):
    """Endless stream of candidates for a tiled BMMC that is not a BPC.

    Each candidate picks k random columns S; rows 0..k-1 on S get a random
    k x k block, rows k..n-1 on S are zero, rows k..n-1 off S get a random
    (n-k) x (n-k) block and rows 0..k-1 off S get random bits.  The caller
    keeps the candidates that are invertible (both blocks invertible).
    """
    g = rng(seed)
    while True:
        cols = sorted(int(v) for v in g.choice(n, size=k, replace=False))
        others = [b for b in range(n) if b not in cols]
        rows = [0] * n
        for r in range(k):
            for b in cols + others:
                if g.integers(0, 2):
                    rows[r] |= 1 << b
        for r in range(k, n):
            for b in others:
                if g.integers(0, 2):
                    rows[r] |= 1 << b
        yield rows


def tiled_only_bmmc(n, k, seed, is_invertible):
    rows = first_passing(tiled_only_candidates(n, k, seed), is_invertible)
    return rows, random_c(n, seed)


# ---------------------------------------------------------------------------
# Payloads: element values unique per index, so any misplacement shows up.
# ---------------------------------------------------------------------------

def _mix32(x):
    """A fixed 32-bit integer hash (multiply-xorshift), for payload filler."""
    x = (x ^ (x >> np.uint64(16))) * np.uint64(0x7FEB352D)
    x &= np.uint64(0xFFFFFFFF)
    x = (x ^ (x >> np.uint64(15))) * np.uint64(0x846CA68B)
    x &= np.uint64(0xFFFFFFFF)
    return x ^ (x >> np.uint64(16))


def payload(n, e, seed=0):
    """A numpy buffer of 2^n elements of e bytes with unique element values.

    e = 4:  uint32 index i
    e = 8:  uint64 i XOR (seed << 32)
    e = 16: four uint32 words (i, ~i, hash(i), seed), shape (2^n, 4)
    """
    count = 1 << n
    i = np.arange(count, dtype=np.uint64)
    if e == 4:
        return i.astype(np.uint32)
    if e == 8:
        return i ^ np.uint64((seed & 0xFFFFFFFF) << 32)
    if e == 16:
        out = np.empty((count, 4), dtype=np.uint32)
        out[:, 0] = i.astype(np.uint32)
        out[:, 1] = (~i).astype(np.uint32)
        out[:, 2] = _mix32(i).astype(np.uint32)
        out[:, 3] = np.uint32(seed & 0xFFFFFFFF)
        return out
    raise ValueError("element size must be 4, 8 or 16 bytes")


def payload_torch(n, e, seed=0, device="cuda"):
    """The same values as ``payload``, generated on a torch device.

    Returned as an int32 tensor of shape (2^n * e / 4,) so that every element
    size shares one dtype for raw byte movement.
    """
    import torch

    count = 1 << n
    i = torch.arange(count, dtype=torch.int64, device=device)
    if e == 4:
        return i.to(torch.int32)
    if e == 8:
        hi = torch.full((count,), seed & 0xFFFFFFFF, dtype=torch.int64,
                        device=device)
        lo = i & 0xFFFFFFFF
        words = torch.stack([lo, hi], dim=1)
        words = torch.where(words >= (1 << 31), words - (1 << 32), words)
        return words.to(torch.int32).reshape(-1)
    if e == 16:
        m = (1 << 32) - 1
        x = i & m
        x = ((x ^ (x >> 16)) * 0x7FEB352D) & m
        x = ((x ^ (x >> 15)) * 0x846CA68B) & m
        h = x ^ (x >> 16)
        words = torch.stack([i & m, (~i) & m, h,
                             torch.full_like(i, seed & m)], dim=1)
        words = torch.where(words >= (1 << 31), words - (1 << 32), words)
        return words.to(torch.int32).reshape(-1)
    raise ValueError("element size must be 4, 8 or 16 bytes")


# ---------------------------------------------------------------------------
# Workload recipes of the benchmark configurations
# ---------------------------------------------------------------------------

def batched_sizes(count=4096, lo=10, hi=24, seed=7):
    """n for each array of the batched workload: n uniform in [lo, hi], so the
    array size 2^n is log-uniform."""
    g = rng(seed)
    return [int(v) for v in g.integers(lo, hi + 1, size=count)]


def serving_requests(rate=2000.0, seconds=10.0, seed=11, n_lo=12, n_hi=27,
                     bp_fraction=0.2):
    """Poisson request stream: list of dicts with arrival time (s), n, e,
    kind ('bp' or 'dense') and a per-request seed."""
    g = rng(seed)
    t = 0.0
    out = []
    idx = 0
    while True:
        t += float(g.exponential(1.0 / rate))
        if t >= seconds:
            break
        out.append({
            "arrival": t,
            "n": int(g.integers(n_lo, n_hi + 1)),
            "e": 4 if g.integers(0, 2) == 0 else 8,
            "kind": "bp" if g.random() < bp_fraction else "dense",
            "seed": 1000 + idx,
        })
        idx += 1
    return out
