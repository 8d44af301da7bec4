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


def _build(tmp_path):
    import paper_2306_07795_gb300 as bm
    bm.lib()  # builds libbmmc.so if needed
    exe = str(tmp_path / "abi_roundtrip")
    cmd = [_nvcc(), "-O2", "-I", os.path.join(ROOT, "include"),
           SRC, "-L", LIBDIR, "-lbmmc", "-Xlinker", "-rpath," + LIBDIR, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


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
