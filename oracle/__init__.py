"""CPU oracle for BMMC permutations -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
The library product never imports, links or executes anything here, and this
package imports nothing from the product.

Two halves:

* ``oracle.f2`` -- plain-Python F2 algebra and the paper's definitions
  (BMMC map, composition, inverse, tiled test, UL.P factorisation, parm,
  stitch functions).
* the C loop in ``bmmc_ref.c`` -- ``out[A x + c] = in[x]`` over every x, for
  arrays too large for Python loops.  ``build_c()`` compiles it with gcc.

Parity of every function is pinned by ``tests/test_oracle_pins.py`` against
values the paper prints, closed forms, and brute force on small inputs.
"""

import ctypes
import os
import subprocess

import numpy as np

from . import f2  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bmmc_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbmmc_ref.so")
_lib = None


def build_c(force=False):
    """Compile bmmc_ref.c into a shared library (gcc, OpenMP if available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_c())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.bmmc_ref_index.restype = ctypes.c_uint64
        lib.bmmc_ref_index.argtypes = [ctypes.c_int, u64p, ctypes.c_uint64,
                                       ctypes.c_uint64]
        for name in ("bmmc_ref_apply", "bmmc_ref_apply_mt", "bmmc_ref_grad"):
            fn = getattr(lib, name)
            fn.restype = None
            fn.argtypes = [ctypes.c_int, u64p, ctypes.c_uint64, ctypes.c_size_t,
                           ctypes.c_void_p, ctypes.c_void_p]
        lib.bmmc_ref_count_mismatch.restype = ctypes.c_uint64
        lib.bmmc_ref_count_mismatch.argtypes = [
            ctypes.c_int, u64p, ctypes.c_uint64, ctypes.c_size_t,
            ctypes.c_void_p, ctypes.c_void_p]
        lib.bmmc_ref_num_threads.restype = ctypes.c_int
        lib.bmmc_ref_num_threads.argtypes = []
        _lib = lib
    return _lib


def _rows_arg(rows):
    arr = (ctypes.c_uint64 * max(1, len(rows)))(*[int(r) for r in rows])
    return arr


def _check_buf(arr, n, e):
    assert arr.flags["C_CONTIGUOUS"]
    assert arr.nbytes == (1 << n) * e, (arr.nbytes, n, e)


def index(n, rows, c, x):
    """A x + c for one index x (C loop)."""
    return int(_load().bmmc_ref_index(n, _rows_arg(rows), c, x))


def apply(n, rows, c, arr, elem_bytes=None, threads=True):
    """out[A x + c] = in[x] over a contiguous numpy buffer of 2^n elements.

    ``elem_bytes`` defaults to the size of one row of ``arr`` along axis 0,
    so an (2^n, 4) uint32 array is treated as 16-byte elements.
    """
    e = elem_bytes or (arr.nbytes >> n)
    _check_buf(arr, n, e)
    out = np.empty_like(arr)
    fn = _load().bmmc_ref_apply_mt if threads else _load().bmmc_ref_apply
    fn(n, _rows_arg(rows), c, e, arr.ctypes.data, out.ctypes.data)
    return out


def apply_into(n, rows, c, arr, out, elem_bytes=None, threads=True):
    """As ``apply``, writing into the preallocated contiguous buffer ``out``
    (the same size as ``arr``), so that a timed loop allocates nothing."""
    e = elem_bytes or (arr.nbytes >> n)
    _check_buf(arr, n, e)
    _check_buf(out, n, e)
    fn = _load().bmmc_ref_apply_mt if threads else _load().bmmc_ref_apply
    fn(n, _rows_arg(rows), c, e, arr.ctypes.data, out.ctypes.data)
    return out


def grad(n, rows, c, gy, elem_bytes=None):
    """gx[x] = gy[A x + c]: the gradient of the forward permutation."""
    e = elem_bytes or (gy.nbytes >> n)
    _check_buf(gy, n, e)
    gx = np.empty_like(gy)
    _load().bmmc_ref_grad(n, _rows_arg(rows), c, e, gy.ctypes.data,
                          gx.ctypes.data)
    return gx


def count_mismatch(n, rows, c, inp, out, elem_bytes=None):
    """Number of x with out[A x + c] != in[x], compared byte by byte."""
    e = elem_bytes or (inp.nbytes >> n)
    _check_buf(inp, n, e)
    _check_buf(out, n, e)
    return int(_load().bmmc_ref_count_mismatch(
        n, _rows_arg(rows), c, e, inp.ctypes.data, out.ctypes.data))


def num_threads():
    """Threads the C loops use (OpenMP), for reporting CPU baselines."""
    return int(_load().bmmc_ref_num_threads())
