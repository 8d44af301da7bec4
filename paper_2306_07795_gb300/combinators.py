"""Array combinators built on BMMC permutations (Sec. 3 and Sec. 6).

parm(mask, f, x): split the last dimension of x (2^n elements) into the two
sub-arrays of the indices i with i . mask = 0 and = 1 (F2 dot product), each
in its original order, apply f to both, and put the results back (Sec. 6.1).
It is computed as Sec. 6.2 prescribes:

    parm mask f = bmmc(A^{-1}, 0) o parm 2^{n-1} f o bmmc(A, 0)

so f always sees the two sub-arrays as the contiguous halves of a
[..., 2, 2^{n-1}] tensor, and both permutations are single library calls.

Pipeline: a sequence of permutations and tensor functions in which adjacent
permutations are fused into one plan by the fusion rule
bmmc(A, c) o bmmc(B, d) = bmmc(A B, A d + c) (Sec. 3), so a chain of k
permutations costs one pass (or two) instead of k.
"""

from . import _binding as B
from .autograd import bmmc_permute
from .plan import Plan


def parm_matrix(n, mask):
    """The matrix A of Sec. 6.2 (row masks), from the library."""
    return B.bmmc_parm_matrix(n, mask)


def _log2_len(x):
    m = x.shape[-1]
    n = m.bit_length() - 1
    if m != 1 << n or n < 1:
        raise ValueError("last dimension must be a power of two >= 2")
    return n


_parm_plans = {}  # (n, mask, element bytes, flags) -> Plan, most recent last
_PARM_PLANS_MAX = 256


def _parm_plan(n, mask, elem_bytes, flags):
    """The plan of parm's permutation, kept for repeated calls (plans are
    immutable; the least recently used one is dropped beyond 256)."""
    key = (n, mask, elem_bytes, flags)
    plan = _parm_plans.pop(key, None)
    if plan is None:
        plan = Plan(n, parm_matrix(n, mask), 0, elem_bytes, flags=flags)
        if len(_parm_plans) >= _PARM_PLANS_MAX:
            _parm_plans.pop(next(iter(_parm_plans)))
    _parm_plans[key] = plan
    return plan


def parm(mask, f, x, flags=B.BMMC_PLAN_PAPER):
    """parm mask f x along the last dimension (differentiable).

    f receives a tensor of shape [..., 2, 2^(n-1)] (the two sub-arrays) and
    must return one of the same shape."""
    n = _log2_len(x)
    plan = _parm_plan(n, mask, x.element_size(), flags)
    y = bmmc_permute(x, plan)
    half = x.shape[-1] // 2
    z = f(y.reshape(*x.shape[:-1], 2, half))
    if tuple(z.shape) != tuple(x.shape[:-1]) + (2, half):
        raise ValueError("f must preserve the shape of the sub-arrays")
    return bmmc_permute(z.reshape(x.shape), plan.inverse())


class Pipeline:
    """Permutations and functions applied left to right to the last dim.

        p = Pipeline(n).perm(rows1, c1).perm(rows2, c2).map(fn).perm(rows3)
        y = p(x)

    Runs of adjacent permutations are fused into one plan per element size
    (cached), by the library's bmmc_plan_compose."""

    def __init__(self, n, flags=B.BMMC_PLAN_PAPER):
        self.n = n
        self.flags = flags
        self.steps = []  # ("perm", rows, c) | ("map", fn)
        self._cache = {}

    def perm(self, rows, c=0):
        if len(rows) != self.n:
            raise ValueError("matrix must have n rows")
        self.steps.append(("perm", [int(r) for r in rows], int(c)))
        self._cache.clear()
        return self

    def parm_perm(self, mask):
        """The (A, 0) of parm mask (its inverse is .perm of the inverse)."""
        return self.perm(parm_matrix(self.n, mask), 0)

    def map(self, fn):
        self.steps.append(("map", fn))
        self._cache.clear()
        return self

    def fused(self, elem_bytes):
        """The step list with each run of permutations fused into one Plan."""
        key = elem_bytes
        if key in self._cache:
            return self._cache[key]
        out = []
        run = None
        for st in self.steps:
            if st[0] == "perm":
                p = Plan(self.n, st[1], st[2], elem_bytes, flags=self.flags)
                if run is None:
                    run = p
                else:
                    h = B.bmmc_plan_compose(p.handle, run.handle)
                    rows, c = B.bmmc_plan_matrix(h, self.n)
                    run = Plan(self.n, rows, c, elem_bytes, flags=self.flags, _handle=h)
            else:
                if run is not None:
                    out.append(("perm", run))
                    run = None
                out.append(st)
        if run is not None:
            out.append(("perm", run))
        self._cache[key] = out
        return out

    def num_permutations(self, elem_bytes=4):
        return sum(1 for st in self.fused(elem_bytes) if st[0] == "perm")

    def __call__(self, x):
        for st in self.fused(x.element_size()):
            if st[0] == "perm":
                x = bmmc_permute(x, st[1])
            else:
                x = st[1](x)
        return x
