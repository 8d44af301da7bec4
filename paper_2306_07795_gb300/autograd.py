"""Differentiable BMMC permutation along the last dimension of a tensor.

Forward: y[..., A i + c] = x[..., i] for every index i of the last dimension
(2^n elements).  A permutation is linear with a 0/1 Jacobian, so the
gradient of any loss L with respect to x is dL/dx[..., i] = dL/dy[..., A i + c]:
the inverse BMMC (A^{-1}, A^{-1} c) applied to the output gradient (the
inverse follows from Sec. 3's definition and fusion rule).  Both directions run
the library's kernels; nothing is computed in PyTorch.

When the leading dimensions hold 2^b rows in total, the whole tensor is one
array of 2^(n+b) elements and the permutation is the BMMC diag(A, I_b) with
complement (c, 0): one launch (or one plan's passes) for the whole batch.
"""

from . import _binding as B
from .plan import Plan

_lift_cache = {}


def _lifted_plan(plan, rows_total):
    b = rows_total.bit_length() - 1
    if rows_total != 1 << b:
        return None
    key = (id(plan), b)
    hit = _lift_cache.get(key)
    if hit is not None and hit[0] is plan:
        return hit[1]
    lifted = plan.lift(b)
    _lift_cache[key] = (plan, lifted)
    return lifted


def _apply(plan, x):
    import torch

    x = x.contiguous()
    last = x.shape[-1] * x.element_size()
    if last != plan.nbytes:
        raise ValueError("last dimension holds %d bytes, the plan needs %d"
                         % (last, plan.nbytes))
    rows_total = x.numel() // x.shape[-1]
    lifted = _lifted_plan(plan, rows_total) if rows_total > 1 else plan
    if lifted is not None:
        return lifted(x.view(-1)).view(x.shape)
    out = torch.empty_like(x)
    xf, of = x.view(rows_total, -1), out.view(rows_total, -1)
    for r in range(rows_total):
        plan(xf[r], out=of[r])
    return out


class BMMCPermute:
    """torch.autograd.Function (built lazily so that importing this module
    does not import torch)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, plan):
                    ctx.plan = plan
                    return _apply(plan, x)

                @staticmethod
                def backward(ctx, gy):
                    return _apply(ctx.plan.inverse(), gy), None

            cls._fn = _Fn
        return cls._fn


def bmmc_permute(x, plan):
    """Differentiable y with y[..., A i + c] = x[..., i] (last dimension)."""
    return BMMCPermute.function().apply(x, plan)


def make_plan(n, rows, c, dtype_bytes, **kw):
    """Plan for permuting a last dimension of 2^n elements of dtype_bytes."""
    return Plan(n, rows, c, dtype_bytes, **kw)


__all__ = ["bmmc_permute", "BMMCPermute", "make_plan", "B"]
