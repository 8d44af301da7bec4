"""Permute-and-compare passes (bmmc_execute_ce) and the Sec. 6.1 sorting
network on the GPU, against the oracle and numpy's sort."""

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300.sorting import SortingNetwork
import workloads as wl

pytestmark = pytest.mark.gpu

KEYS = [("int32", bm._binding.BMMC_KEY_I32, np.int32),
        ("float32", bm._binding.BMMC_KEY_F32, np.float32),
        ("int64", bm._binding.BMMC_KEY_I64, np.int64),
        ("float64", bm._binding.BMMC_KEY_F64, np.float64),
        ("uint32", bm._binding.BMMC_KEY_U32, np.uint32),
        ("uint64", bm._binding.BMMC_KEY_U64, np.uint64)]


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _ce_ref(a):
    """Reference comparator column: keep a pair when a <= b, else swap."""
    a = a.copy()
    lo, hi = a[0::2].copy(), a[1::2].copy()
    swap = ~(lo <= hi)
    a[0::2] = np.where(swap, hi, lo)
    a[1::2] = np.where(swap, lo, hi)
    return a


def _values(np_dtype, count, seed):
    g = wl.rng(seed)
    if np.issubdtype(np_dtype, np.floating):
        v = (g.standard_normal(count) * 100).astype(np_dtype)
        v[::17] = np.nan
        v[3::19] = -0.0
        v[5::23] = 0.0
        v[7::29] = np.inf
        return v
    info = np.iinfo(np_dtype)
    return g.integers(info.min, info.max, size=count, dtype=np_dtype, endpoint=True)


@pytest.mark.parametrize("name,key,np_dtype", KEYS)
@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_execute_ce_matches_reference(name, key, np_dtype, flags):
    import torch
    e = np.dtype(np_dtype).itemsize
    for n in (3, 6, 9, 14, 19):
        rows, c = wl.dense_bmmc(n, 30 + n, _inv)
        arr = _values(np_dtype, 1 << n, n)
        want = _ce_ref(oracle.apply(n, rows, c, arr, elem_bytes=e))
        p = bm.Plan(n, rows, c, e, flags=flags)
        x = torch.from_numpy(arr.view(np.int32 if e == 4 else np.int64).copy()).cuda()
        y = torch.empty_like(x)
        ws = torch.empty(max(p.workspace_bytes, 16), dtype=torch.uint8, device="cuda")
        bm.bmmc_execute_ce(p.handle, x.data_ptr(), y.data_ptr(), ws.data_ptr(), key,
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = y.cpu().numpy().view(np_dtype)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (name, n)


def test_execute_ce_rejects_mismatched_key():
    import torch
    p = bm.Plan(10, wl.bit_reverse(10), 0, 4)
    x = torch.zeros(1 << 10, dtype=torch.int32, device="cuda")
    y = torch.zeros_like(x)
    for key in (0, 4, 7):
        with pytest.raises(bm.BmmcError) as ei:
            bm.bmmc_execute_ce(p.handle, x.data_ptr(), y.data_ptr(), None, key, 0)
        assert ei.value.code == bm.BMMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("dtype_name", ["int32", "float32", "int64", "float64"])
def test_sorting_network_sorts(dtype_name):
    import torch
    dtype = getattr(torch, dtype_name)
    for n in list(range(1, 13)) + [16, 20]:
        g = torch.Generator(device="cuda").manual_seed(n)
        if dtype.is_floating_point:
            x = torch.randn(1 << n, device="cuda", generator=g).to(dtype) * 1000
        else:
            x = torch.randint(-2**30, 2**30, (1 << n,), device="cuda", generator=g).to(dtype)
        got = SortingNetwork(n)(x)
        assert torch.equal(got, torch.sort(x).values), (dtype_name, n)


def test_sorting_network_rows_and_oracle_recursion():
    import torch
    n = 6
    net = SortingNetwork(n)
    assert net.num_stages == n * (n + 1) // 2
    x = torch.randint(-100, 100, (8, 1 << n), dtype=torch.int32, device="cuda")
    got = net(x)
    assert torch.equal(got, torch.sort(x, dim=-1).values)
    for r in range(8):
        xs = x[r].cpu().tolist()
        assert got[r].cpu().tolist() == f2.sort_network(n, xs)


def test_sorting_network_graph_replay():
    import torch
    n = 14
    net = SortingNetwork(n)
    x = torch.randn(1 << n, device="cuda")
    graph, out = net.capture(x)
    for seed in range(3):
        x.copy_(torch.randn(1 << n, device="cuda", generator=torch.Generator(
            device="cuda").manual_seed(seed)))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, torch.sort(x).values)


@pytest.mark.parametrize("name,key,np_dtype", [KEYS[2], KEYS[1]])
def test_execute_ce_full_size(name, key, np_dtype):
    """A permute-and-compare pass at the benchmark's array size (n = 28 at 4
    bytes, n = 27 at 8), dense matrix, both strategies: every element."""
    import torch
    e = np.dtype(np_dtype).itemsize
    n = 28 if e == 4 else 27
    rows, c = wl.dense_bmmc(n, 7, _inv)
    arr = _values(np_dtype, 1 << n, 11)
    want = _ce_ref(oracle.apply(n, rows, c, arr, elem_bytes=e))
    x = torch.from_numpy(arr.view(np.int32 if e == 4 else np.int64).copy()).cuda()
    for flags in (bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS):
        p = bm.Plan(n, rows, c, e, flags=flags)
        y = torch.empty_like(x)
        ws = torch.empty(max(p.workspace_bytes, 16), dtype=torch.uint8, device="cuda")
        bm.bmmc_execute_ce(p.handle, x.data_ptr(), y.data_ptr(), ws.data_ptr(), key,
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = y.cpu().numpy().view(np_dtype)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (name, flags)
        del y, ws


def test_sorting_network_n24():
    import torch
    g = torch.Generator(device="cuda").manual_seed(24)
    x = torch.randn(1 << 24, device="cuda", generator=g)
    assert torch.equal(SortingNetwork(24)(x), torch.sort(x).values)
