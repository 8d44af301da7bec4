"""ctypes binding of the C ABI in include/bmmc.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The library
must be built (``build.build()``); there is no fallback of any kind: if the
shared library is missing or fails to load, importing the package's GPU entry
points raises.
"""

import ctypes
import json
import os

from . import build as _build

BMMC_OK = 0
BMMC_ERR_INVALID = -1
BMMC_ERR_SINGULAR = -2
BMMC_ERR_UNSUPPORTED = -3
BMMC_ERR_ALIAS = -4
BMMC_ERR_ALIGN = -5
BMMC_ERR_OOM = -6
BMMC_ERR_CUDA = -7
BMMC_ERR_TOO_LARGE = -8
BMMC_STATIC_SCRATCH_BYTES = 32 << 20

BMMC_PLAN_PAPER = 0
BMMC_PLAN_SINGLE_PASS = 1
BMMC_PLAN_TMA_LOAD = 2

# Every entry point declared in include/bmmc.h (checked by the tests).
EXPORTED = (
    "bmmc_plan_create", "bmmc_plan_create_ex", "bmmc_plan_destroy",
    "bmmc_plan_num_passes", "bmmc_plan_matrix", "bmmc_plan_pass_matrix",
    "bmmc_plan_inverse",
    "bmmc_plan_workspace_bytes", "bmmc_execute", "bmmc_execute_ws", "bmmc_execute_host",
    "bmmc_execute_static_ws", "bmmc_plan_verify", "bmmc_plan_describe",
    "bmmc_strerror", "bmmc_plan_compose", "bmmc_parm_matrix", "bmmc_execute_ce",
    "bmmc_plan_lift", "bmmc_sort_schedule", "bmmc_device_wait_timeouts",
    # include/bmmc_sort.h
    "bmmc_sort_plan_create", "bmmc_sort_plan_destroy", "bmmc_sort_plan_num_passes",
    "bmmc_sort_workspace_bytes", "bmmc_sort_execute", "bmmc_sort_plan_emulate",
    "bmmc_sort_plan_describe",
    # include/bmmc_shard.h
    "bmmc_shard_plan_create", "bmmc_shard_plan_destroy", "bmmc_shard_plan_num_steps",
    "bmmc_shard_plan_step", "bmmc_shard_plan_verify",
    # include/bmmc_batch.h
    "bmmc_batch_workspace_bytes", "bmmc_batch_table_bytes", "bmmc_batch_create",
    "bmmc_batch_execute",
    "bmmc_batch_num_launches", "bmmc_batch_describe", "bmmc_batch_destroy",
    "bmmc_execute_batch",
    # include/bmmc_debug.h
    "bmmc_debug_fail_allocs", "bmmc_debug_fail_launches",
    # include/bmmc_server.h
    "bmmc_server_create", "bmmc_server_submit", "bmmc_server_drain",
    "bmmc_server_results", "bmmc_server_release", "bmmc_server_stats",
    "bmmc_server_destroy", "bmmc_server_hold", "bmmc_server_now_ms",
)

BMMC_SERVER_CONTINUOUS = 0
BMMC_SERVER_PLAIN = 1


class bmmc_server_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("streams", ctypes.c_int),
                ("budget_bytes", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                ("plan_flags", ctypes.c_uint32), ("group_max_bytes", ctypes.c_uint64),
                ("group_min", ctypes.c_int), ("keep_outputs", ctypes.c_int),
                ("plan_cache", ctypes.c_int), ("large_log2", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


class bmmc_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int),
                ("submit_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("out", ctypes.c_void_p)]


class BmmcError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = lib().bmmc_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, code))


class bmmc_sort_options(ctypes.Structure):
    _fields_ = [("block_log2", ctypes.c_int), ("compare_code", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


class bmmc_plan_options(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("seg_bits", ctypes.c_int),
                ("cta_tile_log2", ctypes.c_int), ("tile_order", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libbmmc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libbmmc.so is missing: the CUDA library was not built")
    L = ctypes.CDLL(path)
    vp, u64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)
    vpp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "bmmc_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, u64p,
                                            ctypes.c_uint64, ctypes.c_size_t]),
        "bmmc_plan_create_ex": (ctypes.c_int,
                                [ctypes.POINTER(vp), ctypes.c_int, u64p,
                                 ctypes.c_uint64, ctypes.c_size_t,
                                 ctypes.POINTER(bmmc_plan_options)]),
        "bmmc_plan_destroy": (None, [vp]),
        "bmmc_plan_num_passes": (ctypes.c_int, [vp]),
        "bmmc_plan_matrix": (ctypes.c_int, [vp, u64p, u64p]),
        "bmmc_plan_pass_matrix": (ctypes.c_int, [vp, ctypes.c_int, u64p, u64p]),
        "bmmc_plan_inverse": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
        "bmmc_plan_workspace_bytes": (ctypes.c_size_t, [vp]),
        "bmmc_execute": (ctypes.c_int, [vp, vp, vp, vp]),
        "bmmc_execute_ws": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bmmc_execute_host": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "bmmc_execute_static_ws": (ctypes.c_int, [vp, vp, vp, vp]),
        "bmmc_plan_verify": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "bmmc_plan_describe": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "bmmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "bmmc_plan_compose": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp)]),
        "bmmc_execute_ce": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, vp]),
        "bmmc_parm_matrix": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, u64p]),
        "bmmc_plan_lift": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp)]),
        "bmmc_device_wait_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong)]),
        "bmmc_sort_schedule": (ctypes.c_int, [ctypes.c_int, u64p, ctypes.c_int, u64p,
                                              ctypes.POINTER(ctypes.c_int)]),
        "bmmc_sort_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(bmmc_sort_options)]),
        "bmmc_sort_plan_destroy": (None, [vp]),
        "bmmc_sort_plan_num_passes": (ctypes.c_int, [vp]),
        "bmmc_sort_workspace_bytes": (ctypes.c_size_t, [vp]),
        "bmmc_sort_execute": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bmmc_sort_plan_emulate": (ctypes.c_int, [vp, vp, vp]),
        "bmmc_sort_plan_describe": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "bmmc_shard_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int,
                                                  ctypes.c_int, u64p, ctypes.c_uint64]),
        "bmmc_shard_plan_destroy": (None, [vp]),
        "bmmc_shard_plan_num_steps": (ctypes.c_int, [vp]),
        "bmmc_shard_plan_step": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_int), u64p, u64p]),
        "bmmc_shard_plan_verify": (ctypes.c_int, [vp]),
        "bmmc_batch_workspace_bytes": (ctypes.c_size_t, [vpp, ctypes.c_int]),
        "bmmc_batch_table_bytes": (ctypes.c_size_t, [vpp, ctypes.c_int]),
        "bmmc_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), vpp, ctypes.c_int,
                                             vpp, vpp, vp, vp, vp]),
        "bmmc_batch_execute": (ctypes.c_int, [vp, vp]),
        "bmmc_batch_num_launches": (ctypes.c_int, [vp]),
        "bmmc_batch_describe": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "bmmc_batch_destroy": (None, [vp]),
        "bmmc_execute_batch": (ctypes.c_int, [vpp, vpp, vpp, ctypes.c_int, vp]),
        "bmmc_debug_fail_allocs": (None, [ctypes.c_int]),
        "bmmc_debug_fail_launches": (None, [ctypes.c_int]),
        "bmmc_server_create": (ctypes.c_int, [ctypes.POINTER(vp),
                                              ctypes.POINTER(bmmc_server_config)]),
        "bmmc_server_submit": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_int, u64p,
                                              ctypes.c_uint64, ctypes.c_size_t, vp]),
        "bmmc_server_drain": (ctypes.c_int, [vp]),
        "bmmc_server_results": (ctypes.c_int, [vp, ctypes.POINTER(bmmc_server_result),
                                               ctypes.c_int]),
        "bmmc_server_release": (ctypes.c_int, [vp, vp]),
        "bmmc_server_stats": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "bmmc_server_destroy": (None, [vp]),
        "bmmc_server_hold": (ctypes.c_int, [vp, ctypes.c_int]),
        "bmmc_server_now_ms": (ctypes.c_double, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(code, what):
    if code != BMMC_OK:
        raise BmmcError(code, what)


def _rows(rows):
    """Row masks as a C uint64 array (an array already converted is passed
    through, so callers on a hot path can convert once)."""
    if isinstance(rows, ctypes.Array):
        return rows
    return (ctypes.c_uint64 * max(1, len(rows)))(*[int(r) for r in rows])


def rows_array(rows):
    """Convert row masks once for repeated calls (see _rows)."""
    return _rows(rows)


# ---------------------------------------------------------------------------
# Functions with the C names
# ---------------------------------------------------------------------------

def bmmc_plan_create(n, rows, c, elem_bytes):
    h = ctypes.c_void_p()
    _check(lib().bmmc_plan_create(ctypes.byref(h), n, _rows(rows), c, elem_bytes),
           "bmmc_plan_create")
    return h


def bmmc_plan_create_ex(n, rows, c, elem_bytes, flags=0, seg_bits=0,
                        cta_tile_log2=0, tile_order=0):
    h = ctypes.c_void_p()
    o = bmmc_plan_options(flags, seg_bits, cta_tile_log2, tile_order)
    _check(lib().bmmc_plan_create_ex(ctypes.byref(h), n, _rows(rows), c,
                                     elem_bytes, ctypes.byref(o)),
           "bmmc_plan_create_ex")
    return h


def bmmc_plan_destroy(h):
    lib().bmmc_plan_destroy(h)


def bmmc_plan_num_passes(h):
    return lib().bmmc_plan_num_passes(h)


def bmmc_plan_matrix(h, n):
    rows = (ctypes.c_uint64 * n)()
    c = ctypes.c_uint64()
    _check(lib().bmmc_plan_matrix(h, rows, ctypes.byref(c)), "bmmc_plan_matrix")
    return [int(r) for r in rows], int(c.value)


def bmmc_plan_pass_matrix(h, n, pass_index):
    rows = (ctypes.c_uint64 * n)()
    c = ctypes.c_uint64()
    _check(lib().bmmc_plan_pass_matrix(h, pass_index, rows, ctypes.byref(c)),
           "bmmc_plan_pass_matrix")
    return [int(r) for r in rows], int(c.value)


def bmmc_plan_inverse(h):
    out = ctypes.c_void_p()
    _check(lib().bmmc_plan_inverse(h, ctypes.byref(out)), "bmmc_plan_inverse")
    return out


def bmmc_plan_workspace_bytes(h):
    return int(lib().bmmc_plan_workspace_bytes(h))


def bmmc_execute(h, in_ptr, out_ptr, stream=0):
    _check(lib().bmmc_execute(h, in_ptr, out_ptr, stream), "bmmc_execute")


def bmmc_execute_ws(h, in_ptr, out_ptr, ws_ptr, stream=0):
    _check(lib().bmmc_execute_ws(h, in_ptr, out_ptr, ws_ptr, stream),
           "bmmc_execute_ws")


def bmmc_execute_host(h, host_in, host_out, dev_in, dev_out, ws_ptr=None, stream=0):
    _check(lib().bmmc_execute_host(h, host_in, host_out, dev_in, dev_out, ws_ptr, stream),
           "bmmc_execute_host")


def bmmc_execute_static_ws(h, in_ptr, out_ptr, stream=0):
    _check(lib().bmmc_execute_static_ws(h, in_ptr, out_ptr, stream),
           "bmmc_execute_static_ws")


def bmmc_plan_verify(h, max_ctas=0):
    return lib().bmmc_plan_verify(h, max_ctas)


def bmmc_plan_describe(h):
    need = lib().bmmc_plan_describe(h, None, 0)
    buf = ctypes.create_string_buffer(need + 1)
    lib().bmmc_plan_describe(h, buf, need + 1)
    return json.loads(buf.value.decode())


def bmmc_strerror(code):
    return lib().bmmc_strerror(code).decode()


def bmmc_plan_compose(second, first):
    out = ctypes.c_void_p()
    _check(lib().bmmc_plan_compose(second, first, ctypes.byref(out)), "bmmc_plan_compose")
    return out


BMMC_KEY_I32, BMMC_KEY_U32, BMMC_KEY_F32 = 1, 2, 3
BMMC_KEY_I64, BMMC_KEY_U64, BMMC_KEY_F64 = 4, 5, 6


def bmmc_execute_ce(h, in_ptr, out_ptr, ws_ptr, key_type, stream=0):
    _check(lib().bmmc_execute_ce(h, in_ptr, out_ptr, ws_ptr, key_type, stream),
           "bmmc_execute_ce")


def bmmc_device_wait_timeouts():
    n = ctypes.c_ulonglong()
    _check(lib().bmmc_device_wait_timeouts(ctypes.byref(n)), "bmmc_device_wait_timeouts")
    return int(n.value)


def bmmc_plan_lift(h, b):
    out = ctypes.c_void_p()
    _check(lib().bmmc_plan_lift(h, b, ctypes.byref(out)), "bmmc_plan_lift")
    return out


def bmmc_sort_schedule(n):
    """(stage matrices, final matrix, final is the identity) of the sorting
    network of 2^n keys."""
    count = lib().bmmc_sort_schedule(n, None, 0, None, None)
    _check(min(count, 0), "bmmc_sort_schedule")
    flat = (ctypes.c_uint64 * (count * n))()
    fin = (ctypes.c_uint64 * n)()
    ident = ctypes.c_int()
    got = lib().bmmc_sort_schedule(n, flat, count, fin, ctypes.byref(ident))
    _check(min(got, 0), "bmmc_sort_schedule")
    stages = [[int(r) for r in flat[s * n:(s + 1) * n]] for s in range(count)]
    return stages, [int(r) for r in fin], bool(ident.value)


def bmmc_parm_matrix(n, mask):
    rows = (ctypes.c_uint64 * n)()
    _check(lib().bmmc_parm_matrix(n, mask, rows), "bmmc_parm_matrix")
    return [int(r) for r in rows]


# ---------------------------------------------------------------------------
# include/bmmc_sort.h
# ---------------------------------------------------------------------------

def bmmc_sort_plan_create(n, b, key_type, block_log2=0, compare_code=0):
    h = ctypes.c_void_p()
    o = bmmc_sort_options(block_log2, compare_code)
    _check(lib().bmmc_sort_plan_create(ctypes.byref(h), n, b, key_type, ctypes.byref(o)),
           "bmmc_sort_plan_create")
    return h


def bmmc_sort_plan_destroy(h):
    lib().bmmc_sort_plan_destroy(h)


def bmmc_sort_plan_num_passes(h):
    return lib().bmmc_sort_plan_num_passes(h)


def bmmc_sort_workspace_bytes(h):
    return int(lib().bmmc_sort_workspace_bytes(h))


def bmmc_sort_execute(h, in_ptr, out_ptr, ws_ptr, stream=0):
    _check(lib().bmmc_sort_execute(h, in_ptr, out_ptr, ws_ptr, stream), "bmmc_sort_execute")


def bmmc_sort_plan_emulate(h, in_ptr, out_ptr):
    _check(lib().bmmc_sort_plan_emulate(h, in_ptr, out_ptr), "bmmc_sort_plan_emulate")


def bmmc_sort_plan_describe(h):
    need = lib().bmmc_sort_plan_describe(h, None, 0)
    buf = ctypes.create_string_buffer(need + 1)
    lib().bmmc_sort_plan_describe(h, buf, need + 1)
    return json.loads(buf.value.decode())


# ---------------------------------------------------------------------------
# include/bmmc_shard.h
# ---------------------------------------------------------------------------

BMMC_SHARD_LOCAL = 0
BMMC_SHARD_EXCHANGE = 1


def bmmc_shard_plan_create(n, g, rows, c):
    h = ctypes.c_void_p()
    _check(lib().bmmc_shard_plan_create(ctypes.byref(h), n, g, _rows(rows), c),
           "bmmc_shard_plan_create")
    return h


def bmmc_shard_plan_destroy(h):
    lib().bmmc_shard_plan_destroy(h)


def bmmc_shard_plan_num_steps(h):
    return lib().bmmc_shard_plan_num_steps(h)


def bmmc_shard_plan_step(h, i, rank, nl):
    """(kind, rows, c) of step i on rank `rank`; rows has nl = n - g masks."""
    kind = ctypes.c_int()
    rows = (ctypes.c_uint64 * max(1, nl))()
    c = ctypes.c_uint64()
    _check(lib().bmmc_shard_plan_step(h, i, rank, ctypes.byref(kind), rows, ctypes.byref(c)),
           "bmmc_shard_plan_step")
    if kind.value == BMMC_SHARD_EXCHANGE:
        return kind.value, None, None
    return kind.value, [int(r) for r in rows[:nl]], int(c.value)


def bmmc_shard_plan_verify(h):
    return lib().bmmc_shard_plan_verify(h)


# ---------------------------------------------------------------------------
# include/bmmc_batch.h
# ---------------------------------------------------------------------------

def _ptr_array(values):
    arr = (ctypes.c_void_p * max(1, len(values)))()
    for i, v in enumerate(values):
        arr[i] = v.value if isinstance(v, ctypes.c_void_p) else v
    return arr


def bmmc_batch_workspace_bytes(plan_handles):
    return int(lib().bmmc_batch_workspace_bytes(_ptr_array(plan_handles),
                                                len(plan_handles)))


def bmmc_batch_table_bytes(plan_handles):
    return int(lib().bmmc_batch_table_bytes(_ptr_array(plan_handles),
                                            len(plan_handles)))


def bmmc_batch_create(plan_handles, in_ptrs, out_ptrs, ws_ptr, table_ptr, stream=0):
    h = ctypes.c_void_p()
    _check(lib().bmmc_batch_create(ctypes.byref(h), _ptr_array(plan_handles),
                                   len(plan_handles), _ptr_array(in_ptrs),
                                   _ptr_array(out_ptrs), ws_ptr, table_ptr, stream),
           "bmmc_batch_create")
    return h


def bmmc_batch_execute(h, stream=0):
    _check(lib().bmmc_batch_execute(h, stream), "bmmc_batch_execute")


def bmmc_batch_num_launches(h):
    return lib().bmmc_batch_num_launches(h)


def bmmc_batch_describe(h):
    need = lib().bmmc_batch_describe(h, None, 0)
    buf = ctypes.create_string_buffer(need + 1)
    lib().bmmc_batch_describe(h, buf, need + 1)
    return json.loads(buf.value.decode())


def bmmc_batch_destroy(h):
    lib().bmmc_batch_destroy(h)


def bmmc_debug_fail_allocs(count):
    lib().bmmc_debug_fail_allocs(int(count))


def bmmc_debug_fail_launches(count):
    lib().bmmc_debug_fail_launches(int(count))


def bmmc_execute_batch(plan_handles, in_ptrs, out_ptrs, stream=0):
    _check(lib().bmmc_execute_batch(_ptr_array(plan_handles), _ptr_array(in_ptrs),
                                    _ptr_array(out_ptrs), len(plan_handles), stream),
           "bmmc_execute_batch")


# ---------------------------------------------------------------------------
# include/bmmc_server.h
# ---------------------------------------------------------------------------

def bmmc_server_create(cfg):
    h = ctypes.c_void_p()
    _check(lib().bmmc_server_create(ctypes.byref(h), ctypes.byref(cfg)),
           "bmmc_server_create")
    return h


def bmmc_server_submit(h, rid, n, rows, c, elem_bytes, in_ptr):
    """Returns the status code (a request rejected at submission is not queued)."""
    return lib().bmmc_server_submit(h, rid, n, _rows(rows), c, elem_bytes, in_ptr)


def bmmc_server_drain(h):
    _check(lib().bmmc_server_drain(h), "bmmc_server_drain")


def bmmc_server_results(h, max_results=4096):
    buf = (bmmc_server_result * max_results)()
    out = []
    while True:
        k = lib().bmmc_server_results(h, buf, max_results)
        if k < 0:
            _check(k, "bmmc_server_results")
        out.extend((r.id, r.status, r.submit_ms, r.done_ms, r.out) for r in buf[:k])
        if k < max_results:
            return out


def bmmc_server_release(h, ptr):
    _check(lib().bmmc_server_release(h, ptr), "bmmc_server_release")


def bmmc_server_stats(h):
    need = lib().bmmc_server_stats(h, None, 0)
    buf = ctypes.create_string_buffer(need + 1)
    lib().bmmc_server_stats(h, buf, need + 1)
    return json.loads(buf.value.decode())


def bmmc_server_destroy(h):
    lib().bmmc_server_destroy(h)


def bmmc_server_hold(h, hold):
    _check(lib().bmmc_server_hold(h, 1 if hold else 0), "bmmc_server_hold")


def bmmc_server_now_ms(h):
    return float(lib().bmmc_server_now_ms(h))
