"""parm and fused permutation pipelines on the GPU against the oracle's
definitions (Sec. 6.1 partition definition; Sec. 3 fusion rule)."""

import numpy as np
import pytest

from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300.combinators import Pipeline, parm
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _f_torch(t):
    """Reverse each sub-array and add its length (not symmetric in its input)."""
    return t.flip(-1) + t.shape[-1]


def _f_list(ys):
    return [v + len(ys) for v in reversed(ys)]


@pytest.mark.parametrize("n", [3, 6, 10])
def test_parm_matches_definition(n):
    import torch
    masks = range(1, 1 << n) if n <= 6 else [1, 3, 0b1010101, 1 << (n - 1), (1 << n) - 1]
    xs = list(range(1 << n))
    x = torch.arange(1 << n, dtype=torch.int32, device="cuda")
    for mask in masks:
        want = f2.parm_apply(mask, _f_list, xs)
        got = parm(mask, _f_torch, x)
        assert got.cpu().tolist() == want, mask


def test_parm_batched_and_differentiable():
    import torch
    n = 8
    x = torch.randn(4, 1 << n, dtype=torch.float64, device="cuda", requires_grad=True)
    y = parm(0b10110, lambda t: t * 2.0, x)
    assert torch.equal(y, x * 2.0)  # f acts elementwise: parm is transparent
    y.sum().backward()
    assert torch.equal(x.grad, torch.full_like(x, 2.0))
    # a position-dependent f: gradient flows back through both permutations
    x.grad = None
    w = torch.randn(4, 2, 1 << (n - 1), dtype=torch.float64, device="cuda")
    z = parm(0b10110, lambda t: t * w, x)
    z.sum().backward()
    assert torch.autograd.gradcheck(lambda t: parm(0b11, lambda u: u * w, t),
                                    (x.detach().requires_grad_(True),))


def test_nested_parm_vcolumn():
    """vcolumn n = parm 3 (vcolumn (n - 1)) (Sec. 6.1), with vcolumn 1 ordering a
    pair, built from nested GPU parm calls, against the oracle's recursion."""
    import torch

    def vcol(n, t):
        if n == 1:
            a, b = t[..., 0:1], t[..., 1:2]
            return torch.cat([torch.minimum(a, b), torch.maximum(a, b)], dim=-1)
        return parm(3, lambda u: vcol(n - 1, u), t)

    n = 6
    g = wl.rng(1)
    xs = [int(v) for v in g.integers(-50, 50, size=1 << n)]
    got = vcol(n, torch.tensor(xs, dtype=torch.int32, device="cuda"))
    assert got.cpu().tolist() == f2.vcolumn(n, xs)


def test_pipeline_fusion_on_device():
    import torch
    n = 16
    mats = [wl.dense_bmmc(n, s, _inv) for s in range(4)]
    p = Pipeline(n)
    for rows, c in mats[:3]:
        p.perm(rows, c)
    p.map(lambda t: t + 1)
    p.perm(*mats[3])
    assert p.num_permutations() == 2
    arr = np.arange(1 << n, dtype=np.int32)
    x = torch.from_numpy(arr.copy()).cuda()
    got = p(x).cpu().numpy()
    want = arr
    for rows, c in mats[:3]:
        want = f2.apply(n, rows, c, want)
    want = f2.apply(n, mats[3][0], mats[3][1], want + 1)
    assert np.array_equal(got, want)
