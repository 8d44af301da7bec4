"""The differentiable permutation: forward bit-exact, backward bit-exact
against an explicit scatter reference, and against central finite
differences."""

import numpy as np
import pytest

from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300.autograd import bmmc_permute
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _dest_index(n, rows, c):
    """A i + c for every i (the oracle's numpy evaluation of the definition)."""
    return f2.index_table(n, rows, c).astype(np.int64)


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_gradient_config(flags):
    """[64, 2^20] fp32, x ~ N(0, 1) (seed 3), dense BMMC on the last dim."""
    import torch
    n, rows_b = 20, 64
    rows, c = wl.dense_bmmc(n, 3, _inv)
    plan = bm.Plan(n, rows, c, 4, flags=flags)
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(rows_b, 1 << n, device="cuda", generator=g).requires_grad_(True)
    w = torch.randn(rows_b, 1 << n, device="cuda", generator=g)
    y = bmmc_permute(x, plan)
    dest = torch.from_numpy(_dest_index(n, rows, c)).cuda()
    # forward: y[..., A i + c] = x[..., i]
    y_ref = torch.empty_like(x).scatter_(1, dest.expand(rows_b, -1), x.detach())
    assert torch.equal(y, y_ref)
    loss = (w.double() * y.double()).sum()
    loss.backward()
    gx = x.grad
    # explicit scatter-based reference: output gradient w[..., y] flows back
    # to the input position that was sent to y
    src_of = torch.empty_like(dest).scatter_(0, dest, torch.arange(1 << n, device="cuda"))
    gx_scatter = torch.zeros_like(w).scatter_(1, src_of.expand(rows_b, -1), w)
    assert torch.equal(gx.view(torch.int32), gx_scatter.view(torch.int32))
    gx_gather = w[:, dest]
    assert torch.equal(gx.view(torch.int32), gx_gather.view(torch.int32))

    # central finite differences, eps = 1e-2, loss accumulated in fp64
    def L(xv):
        with torch.no_grad():
            return float((w.double() * bmmc_permute(xv, plan).double()).sum())

    eps = 1e-2
    gen = torch.Generator(device="cuda").manual_seed(5)
    xd = x.detach()
    for _ in range(32):
        v = torch.randn(xd.shape, device="cuda", generator=gen)
        fd = (L(xd + eps * v) - L(xd - eps * v)) / (2 * eps)
        an = float((gx.double() * v.double()).sum())
        assert abs(fd - an) <= 1e-3 * max(1.0, abs(an)), (fd, an)
    idx = torch.randint(0, xd.numel(), (256,), device="cuda", generator=gen)
    for k in idx.tolist():
        v = torch.zeros_like(xd).view(-1)
        v[k] = 1.0
        v = v.view(xd.shape)
        fd = (L(xd + eps * v) - L(xd - eps * v)) / (2 * eps)
        an = float(gx.view(-1)[k])
        assert abs(fd - an) <= 1e-3 * max(1.0, abs(an)), (k, fd, an)


def test_non_power_of_two_rows_and_dtypes():
    import torch
    n = 10
    rows, c = wl.dense_bmmc(n, 9, _inv)
    for dtype, e in ((torch.float32, 4), (torch.float64, 8)):
        plan = bm.Plan(n, rows, c, e)
        x = torch.randn(3, 5, 1 << n, dtype=dtype, device="cuda", requires_grad=True)
        y = bmmc_permute(x, plan)
        dest = torch.from_numpy(_dest_index(n, rows, c)).cuda()
        y_ref = torch.empty_like(x).scatter_(2, dest.expand(3, 5, -1), x.detach())
        assert torch.equal(y, y_ref)
        gy = torch.randn_like(y)
        y.backward(gy)
        assert torch.equal(x.grad, gy[:, :, dest])


def test_gradcheck_small():
    import torch
    n = 6
    rows, c = wl.dense_bmmc(n, 2, _inv)
    plan = bm.Plan(n, rows, c, 8)
    x = torch.randn(4, 1 << n, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: bmmc_permute(t, plan), (x,))


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_forward_backward_graph_capture(flags):
    """Forward and backward captured in one CUDA graph: every replay gives
    the eager result for the inputs written into the static buffers."""
    import torch
    n, rows_b = 12, 8
    rows, c = wl.dense_bmmc(n, 21, _inv)
    plan = bm.Plan(n, rows, c, 4, flags=flags)
    x = torch.randn(rows_b, 1 << n, device="cuda", requires_grad=True)
    w = torch.randn(rows_b, 1 << n, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):  # plans, inverse plans and allocator state
            x.grad = None
            bmmc_permute(x, plan).backward(w)
    torch.cuda.current_stream().wait_stream(s)
    x.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        y = bmmc_permute(x, plan)
        y.backward(w)
    dest = torch.from_numpy(_dest_index(n, rows, c)).cuda()
    for seed in range(3):
        gen = torch.Generator(device="cuda").manual_seed(seed)
        with torch.no_grad():
            x.copy_(torch.randn(x.shape, device="cuda", generator=gen))
            w.copy_(torch.randn(w.shape, device="cuda", generator=gen))
        g.replay()
        torch.cuda.synchronize()
        y_ref = torch.empty_like(w).scatter_(1, dest.expand(rows_b, -1), x.detach())
        assert torch.equal(y, y_ref)
        assert torch.equal(x.grad, w[:, dest])
