"""The library through its C ABI alone: a C program (tests/c/abi_roundtrip.c)
that includes only include/bmmc.h and links libbmmc.so and the CUDA runtime.
Building it checks that the header is valid C and that the library exports
what the program calls; running it (GPU) checks its output against the
oracle."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import f2
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_roundtrip.c")
LIBDIR = os.path.join(ROOT, "paper_2306_07795_gb300", "_lib")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


EXTRAS = os.path.join(ROOT, "tests", "c", "abi_extras.c")


def _build(tmp_path, src=SRC):
    import paper_2306_07795_gb300 as bm
    bm.lib()  # builds libbmmc.so if needed
    exe = str(tmp_path / os.path.splitext(os.path.basename(src))[0])
    cmd = [_nvcc(), "-O2", "-I", os.path.join(ROOT, "include"),
           src, "-L", LIBDIR, "-lbmmc", "-Xlinker", "-rpath," + LIBDIR, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


def test_c_extras_program_builds(tmp_path):
    assert os.path.exists(_build(tmp_path, EXTRAS))


def _job(arrays, payloads=True):
    """The job abi_extras.c reads: headers as uint64 words, then bytes."""
    words = [len(arrays)]
    for n, e, rows, c, _ in arrays:
        words += [n, e, c] + [int(r) for r in rows]
    data = np.array(words, dtype=np.uint64).tobytes()
    if payloads:
        for *_, arr in arrays:
            data += np.ascontiguousarray(arr).reshape(-1).view(np.uint8).tobytes()
    return data


def _run_extras(tmp_path, mode, job):
    r = subprocess.run([_build(tmp_path, EXTRAS), mode], input=job, capture_output=True,
                       timeout=300)
    assert r.returncode == 0, (mode, r.returncode, r.stderr.decode())
    return r.stdout


def test_c_shard_plans(tmp_path):
    """bmmc_shard.h from C (host only): one exchange between two local steps
    for dense matrices, every index checked by bmmc_shard_plan_verify."""
    arrays = []
    for n in (6, 10, 14, 20):
        rows, c = wl.dense_bmmc(n, 30 + n, _inv)
        arrays.append((n, 4, rows, c, None))
    out = np.frombuffer(_run_extras(tmp_path, "shard", _job(arrays, payloads=False)),
                        dtype=np.uint64).reshape(-1, 2)
    assert out.shape == (4, 2)
    assert all(steps in (3, 5) for steps in out[:, 0]) and not out[:, 1].any(), out


def _mixed_arrays():
    arrays = []
    for i, (n, e) in enumerate([(6, 4), (12, 8), (16, 16), (19, 4), (21, 8), (9, 4)]):
        rows, c = wl.dense_bmmc(n, 50 + i, _inv) if i % 2 == 0 else (wl.random_bp(n, i), 0)
        arrays.append((n, e, rows, c, wl.payload(n, e, seed=i)))
    return arrays


def _split(out, arrays):
    pos = 0
    for n, e, rows, c, arr in arrays:
        size = (1 << n) * e
        yield out[pos:pos + size], n, e, rows, c, arr
        pos += size
    assert pos == len(out)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batch", "server"])
def test_c_batch_and_server_match_oracle(tmp_path, mode):
    arrays = _mixed_arrays()
    out = _run_extras(tmp_path, mode, _job(arrays))
    for got, n, e, rows, c, arr in _split(out, arrays):
        want = np.ascontiguousarray(oracle.apply(n, rows, c, arr, elem_bytes=e))
        assert got == want.reshape(-1).view(np.uint8).tobytes(), (mode, n, e)


@pytest.mark.gpu
def test_c_sort_matches_numpy(tmp_path):
    g = wl.rng(12)
    arrays = []
    for n in (5, 12, 13, 17, 23):
        keys = g.integers(-2**31, 2**31 - 1, size=1 << n, dtype=np.int64).astype(np.int32)
        arrays.append((n, 4, [1 << i for i in range(n)], 0, keys))
    out = _run_extras(tmp_path, "sort", _job(arrays))
    for got, n, e, rows, c, keys in _split(out, arrays):
        assert np.array_equal(np.frombuffer(got, dtype=np.int32), np.sort(keys)), n


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


@pytest.mark.gpu
@pytest.mark.parametrize("n,e,kind", [(18, 4, "dense"), (20, 16, "bit_reverse"),
                                      (9, 8, "bp"), (6, 4, "dense"), (17, 8, "dense")])
def test_c_program_matches_oracle(tmp_path, n, e, kind):
    exe = _build(tmp_path)
    if kind == "dense":
        rows, c = wl.dense_bmmc(n, 80 + n, _inv)
    elif kind == "bp":
        rows, c = wl.random_bp(n, 4), 0
    else:
        rows, c = wl.bit_reverse(n), 0
    arr = wl.payload(n, e, seed=3)
    data = np.ascontiguousarray(arr).reshape(-1).view(np.uint8).tobytes()
    args = [exe, str(n), str(e), str(c)] + [str(r) for r in rows]
    r = subprocess.run(args, input=data, capture_output=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr.decode())
    want = np.ascontiguousarray(oracle.apply(n, rows, c, arr, elem_bytes=e))
    assert r.stdout == want.reshape(-1).view(np.uint8).tobytes()
