"""Fused sorting-network passes (include/bmmc_sort.h) on the GPU: bit for bit
the output of the one-pass-per-stage network (bmmc_execute_ce), of the plan's
host emulation, and of the Sec. 6.1 network simulated with the oracle."""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2306_07795_gb300 import _binding as B
from paper_2306_07795_gb300.sorting import SortingNetwork, schedule

pytestmark = pytest.mark.gpu

DT = {"int32": (np.int32, B.BMMC_KEY_I32), "uint32": (np.uint32, B.BMMC_KEY_U32),
      "float32": (np.float32, B.BMMC_KEY_F32), "int64": (np.int64, B.BMMC_KEY_I64),
      "uint64": (np.uint64, B.BMMC_KEY_U64), "float64": (np.float64, B.BMMC_KEY_F64)}


def _keys(np_dtype, count, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    if np.issubdtype(np_dtype, np.floating):
        v = (g.standard_normal(count) * 100).astype(np_dtype)
        v[::17] = np.nan
        v[3::19] = -0.0
        v[5::23] = 0.0
        v[7::29] = np.inf
        v[9::31] = -np.inf
        bits = v.view(np.uint32 if v.itemsize == 4 else np.uint64)
        bits[11::37] |= 1  # NaN payloads differ... and finite values shift by one ulp
        return v
    return g.integers(-1000, 1000, size=count, endpoint=True).astype(np_dtype)


def _to_torch(arr):
    import torch
    word = np.int32 if arr.itemsize == 4 else np.int64
    return torch.from_numpy(arr.view(word).copy()).cuda()


def _run(net, arr, rows):
    import torch
    tdt = {"int32": torch.int32, "float32": torch.float32, "int64": torch.int64,
           "float64": torch.float64, "uint32": getattr(torch, "uint32", None),
           "uint64": getattr(torch, "uint64", None)}[arr.dtype.name]
    if tdt is None:
        pytest.skip("this torch has no %s" % arr.dtype.name)
    x = _to_torch(arr).view(tdt).view(rows, -1)
    y = net(x)
    torch.cuda.synchronize()
    word = torch.int32 if arr.itemsize == 4 else torch.int64
    return y.contiguous().view(word).view(-1).cpu().numpy().view(arr.dtype)


def _ce(a):
    a = a.copy()
    lo, hi = a[0::2].copy(), a[1::2].copy()
    with np.errstate(invalid="ignore"):
        swap = ~(lo <= hi)
    a[0::2] = np.where(swap, hi, lo)
    a[1::2] = np.where(swap, lo, hi)
    return a


def _network(n, row):
    stages, final, _ = schedule(n)
    a = np.ascontiguousarray(row)
    for rows in stages:
        a = _ce(oracle.apply(n, rows, 0, a, elem_bytes=a.itemsize))
    return oracle.apply(n, final, 0, a, elem_bytes=a.itemsize)


@pytest.mark.parametrize("name", ["int32", "float32", "int64", "float64"])
@pytest.mark.parametrize("n,b", [(4, 0), (12, 0), (13, 0), (15, 1), (16, 0), (9, 6)])
def test_fused_equals_stagewise(name, n, b):
    np_dtype, _ = DT[name]
    arr = _keys(np_dtype, 1 << (n + b), n * 31 + b)
    fused = _run(SortingNetwork(n), arr, 1 << b)
    stagewise = _run(SortingNetwork(n, fused=False), arr, 1 << b)
    assert np.array_equal(fused.view(np.uint8), stagewise.view(np.uint8))


@pytest.mark.parametrize("name", ["uint32", "float32", "int64"])
def test_fused_equals_oracle_network(name):
    np_dtype, _ = DT[name]
    n, b = 14, 1
    arr = _keys(np_dtype, 1 << (n + b), 5)
    got = _run(SortingNetwork(n), arr, 1 << b)
    want = np.concatenate([_network(n, r) for r in arr.reshape(1 << b, -1)])
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("n,name,block_log2", [(18, "float32", 0), (20, "float32", 0),
                                               (20, "float64", 0), (19, "int32", 14),
                                               (17, "uint64", 15), (16, "int32", 16),
                                               (19, "uint32", 16), (20, "float32", 16)])
def test_fused_equals_host_emulation(n, name, block_log2):
    """The kernels index shared memory and registers exactly as the host walk
    of the same tables does (bmmc_sort_plan_emulate)."""
    np_dtype, key = DT[name]
    arr = _keys(np_dtype, 1 << n, n)
    h = B.bmmc_sort_plan_create(n, 0, key, block_log2)
    want = np.empty_like(arr)
    B.bmmc_sort_plan_emulate(h, ctypes.c_void_p(arr.ctypes.data),
                             ctypes.c_void_p(want.ctypes.data))
    import torch
    x = _to_torch(arr)
    y = torch.full_like(x, -1)
    ws = torch.empty(max(16, B.bmmc_sort_workspace_bytes(h)), dtype=torch.uint8, device="cuda")
    B.bmmc_sort_execute(h, x.data_ptr(), y.data_ptr(), ws.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    B.bmmc_sort_plan_destroy(h)
    got = y.cpu().numpy().view(np_dtype)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_fused_random_options():
    """Seeded random sizes, row counts, key types, block sizes and compare
    forms: the kernels equal the host emulation of the same plan bit for bit
    (float keys with NaN payloads, infinities and both zeros), and integer
    keys equal numpy's sort row by row."""
    import torch
    g = np.random.Generator(np.random.PCG64(77))
    names = list(DT)
    checked = 0
    for it in range(48):
        name = names[it % len(names)]
        np_dtype, key = DT[name]
        n = int(g.integers(1, 19))
        b = int(g.integers(0, 3))
        block_log2 = int(g.choice([0, 14, 15, 16]))
        compare_code = int(g.choice([0, 1, 2]))
        try:
            h = B.bmmc_sort_plan_create(n, b, key, block_log2, compare_code)
        except B.BmmcError as err:
            assert err.code == B.BMMC_ERR_UNSUPPORTED, (n, b, name, block_log2)
            continue
        arr = _keys(np_dtype, 1 << (n + b), 1000 + it)
        want = np.empty_like(arr)
        B.bmmc_sort_plan_emulate(h, ctypes.c_void_p(arr.ctypes.data),
                                 ctypes.c_void_p(want.ctypes.data))
        x = _to_torch(arr)
        y = torch.full_like(x, -1)
        ws = torch.empty(max(16, B.bmmc_sort_workspace_bytes(h)), dtype=torch.uint8,
                         device="cuda")
        B.bmmc_sort_execute(h, x.data_ptr(), y.data_ptr(), ws.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        B.bmmc_sort_plan_destroy(h)
        got = y.cpu().numpy().view(np_dtype)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), \
            (it, n, b, name, block_log2, compare_code)
        if not np.issubdtype(np_dtype, np.floating):
            assert np.array_equal(got.reshape(1 << b, -1),
                                  np.sort(arr.reshape(1 << b, -1), axis=1)), (it, n, b, name)
        checked += 1
    assert checked >= 30


@pytest.mark.parametrize("n", [20, 24])
def test_fused_matches_torch_sort(n):
    import torch
    g = torch.Generator(device="cuda").manual_seed(n)
    x = torch.randn(1 << n, device="cuda", generator=g)
    assert torch.equal(SortingNetwork(n)(x), torch.sort(x).values)
    xi = torch.randint(-2**31, 2**31 - 1, (4, 1 << (n - 2)), device="cuda", generator=g,
                       dtype=torch.int64)
    assert torch.equal(SortingNetwork(n - 2)(xi), torch.sort(xi, dim=-1).values)


def test_fused_graph_replay():
    import torch
    n = 20
    net = SortingNetwork(n)
    x = torch.randn(1 << n, device="cuda")
    graph, out = net.capture(x)
    for seed in range(3):
        x.copy_(torch.randn(1 << n, device="cuda",
                            generator=torch.Generator(device="cuda").manual_seed(seed)))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, torch.sort(x).values)


def test_fused_argument_errors():
    import torch
    h = B.bmmc_sort_plan_create(16, 0, B.BMMC_KEY_F32)
    assert B.bmmc_sort_workspace_bytes(h) == 4 << 16
    x = torch.zeros(3 << 16, dtype=torch.float32, device="cuda")
    a, b, c = x[: 1 << 16], x[1 << 16: 2 << 16], x[2 << 16:]
    s = torch.cuda.current_stream().cuda_stream
    for args, code in (((a.data_ptr(), a.data_ptr(), b.data_ptr()), B.BMMC_ERR_ALIAS),
                       ((a.data_ptr(), b.data_ptr(), b.data_ptr()), B.BMMC_ERR_ALIAS),
                       ((a.data_ptr(), b.data_ptr(), None), B.BMMC_ERR_INVALID),
                       ((a.data_ptr() + 4, b.data_ptr(), c.data_ptr()), B.BMMC_ERR_ALIGN)):
        with pytest.raises(B.BmmcError) as ei:
            B.bmmc_sort_execute(h, *args, s)
        assert ei.value.code == code
    B.bmmc_sort_execute(h, a.data_ptr(), b.data_ptr(), c.data_ptr(), s)
    torch.cuda.synchronize()
    B.bmmc_sort_plan_destroy(h)
