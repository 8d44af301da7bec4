"""The sorting network of Sec. 6.1, compiled to fused permute-and-compare passes.

The paper writes an even/odd merge sort with a balanced periodic merger in
terms of parm:

    sort n    = merge n  o  parm 1 (sort (n - 1))
    merge n   = parm 2^(n-1) (merge (n - 1))  o  vcolumn n
    vcolumn n = parm 3 (vcolumn (n - 1)),   vcolumn 1 orders a pair

and parm m f = bmmc(A^{-1}) o parm 2^(n-1) f o bmmc(A) (Sec. 6.2), where the
inner f acts on the low n - 1 index bits (the two halves).  Unrolling the
recursion gives a straight program of permutations and comparator columns;
every comparator column compares adjacent pairs (index bit 0), because the
innermost f is vcolumn 1 on two-element arrays.  The fusion rule (Sec. 3)
collapses each run of permutations between two columns into one BMMC, so

    sort n = P_final o CE o P_s o ... o CE o P_1

with n (n + 1) / 2 comparator columns.  Each "CE o P" is one pass of the
library (bmmc_execute_ce: the comparator runs in registers before the
permutation's 16-byte store), and the whole network is a CUDA-graph-friendly
sequence of single-pass launches.

The schedule comes from the library (bmmc_sort_schedule) and the lifted
plans from bmmc_plan_lift; the data path is entirely library kernels.
"""

from . import _binding as B
from .plan import Plan

_KEYS = {}


def _key_for(dtype):
    import torch
    if not _KEYS:
        _KEYS.update({torch.int32: (4, B.BMMC_KEY_I32), torch.float32: (4, B.BMMC_KEY_F32),
                      torch.int64: (8, B.BMMC_KEY_I64), torch.float64: (8, B.BMMC_KEY_F64)})
        if hasattr(torch, "uint32"):
            _KEYS[torch.uint32] = (4, B.BMMC_KEY_U32)
        if hasattr(torch, "uint64"):
            _KEYS[torch.uint64] = (8, B.BMMC_KEY_U64)
    if dtype not in _KEYS:
        raise TypeError("sorting keys must be 32- or 64-bit integers or floats")
    return _KEYS[dtype]


def schedule(n):
    """The fused program of sort n from the library (bmmc_sort_schedule):
    (stage matrices, final matrix, final is the identity).  Stage s is
    'permute by M_s, then order adjacent pairs'."""
    return B.bmmc_sort_schedule(n)


class _SortPlan:
    """Owner of one bmmc_sort_plan handle (fused passes)."""

    def __init__(self, n, b, key, block_log2, compare_code):
        self.h = B.bmmc_sort_plan_create(n, b, key, block_log2, compare_code)
        self.ws_bytes = B.bmmc_sort_workspace_bytes(self.h)
        self.passes = B.bmmc_sort_plan_num_passes(self.h)

    def describe(self):
        return B.bmmc_sort_plan_describe(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None:
            try:
                B.bmmc_sort_plan_destroy(h)
            except Exception:
                pass
            self.h = None


class SortingNetwork:
    """Sorts the last dimension (2^n elements) of int32 / float32 / int64 /
    float64 tensors with the network of Sec. 6.1; leading dimensions holding
    2^b rows are sorted independently in the same passes.

    fused=True (default) runs the network through a sort plan
    (include/bmmc_sort.h): many comparator stages per pass, on tiles held in
    shared memory and registers.  fused=False runs one permute-and-compare
    pass per stage (bmmc_execute_ce), the straightforward form of Sec. 6.1's
    program; both give the same output bit for bit."""

    def __init__(self, n, fused=True, block_log2=0, compare_code=0):
        if n < 1 or n > 30:
            raise ValueError("n must be in 1..30")
        self.n = n
        self.fused = fused
        self.block_log2 = block_log2
        self.compare_code = compare_code
        self.stage_rows, self.final_rows, self._final_identity = schedule(n)
        self._plans = {}

    @property
    def num_stages(self):
        return len(self.stage_rows)

    def num_passes(self, dtype, rows=1):
        """Kernel launches one call makes for `rows` rows of `dtype` keys."""
        import torch
        elem_bytes, key = _key_for(dtype)
        b = rows.bit_length() - 1
        if self.fused:
            return self._sort_plan(key, b).passes
        stages, final = self._plans_for(elem_bytes, b)
        return len(stages) + (final is not None)

    def _sort_plan(self, key, b):
        k = ("fused", key, b)
        if k not in self._plans:
            self._plans[k] = _SortPlan(self.n, b, key, self.block_log2, self.compare_code)
        return self._plans[k]

    def describe(self, dtype, rows=1):
        _, key = _key_for(dtype)
        return self._sort_plan(key, rows.bit_length() - 1).describe()

    def _plans_for(self, elem_bytes, b):
        key = (elem_bytes, b)
        if key not in self._plans:
            def mk(rows):
                return Plan(self.n, rows, 0, elem_bytes,
                            flags=B.BMMC_PLAN_SINGLE_PASS).lift(b)
            stages = [mk(r) for r in self.stage_rows]
            final = None if self._final_identity else mk(self.final_rows)
            self._plans[key] = (stages, final)
        return self._plans[key]

    def capture(self, x):
        """Record the whole network for input buffer x in a CUDA graph.
        Returns (graph, out): after graph.replay(), out holds x sorted (x may be
        refilled between replays; its address is baked into the graph)."""
        import torch
        self(x)  # plans and kernel attributes outside capture
        torch.cuda.synchronize(x.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.device(x.device):
            with torch.cuda.graph(g):
                out = self(x)
        return g, out

    def __call__(self, x, stream=None):
        import torch
        elem_bytes, key = _key_for(x.dtype)
        if not x.is_cuda:
            raise ValueError("x must be a CUDA tensor (there is no CPU path)")
        if x.shape[-1] != 1 << self.n:
            raise ValueError("last dimension must hold 2^n elements")
        rows_total = x.numel() // x.shape[-1]
        b = rows_total.bit_length() - 1
        if rows_total != 1 << b:
            raise ValueError("leading dimensions must hold a power-of-two count of rows")
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        src = x.contiguous()
        if self.fused:
            sp = self._sort_plan(key, b)
            out = torch.empty_like(src)
            ws = torch.empty(sp.ws_bytes, dtype=torch.uint8, device=x.device) \
                if sp.ws_bytes else None
            with torch.cuda.device(x.device):
                B.bmmc_sort_execute(sp.h, src.data_ptr(), out.data_ptr(),
                                    ws.data_ptr() if ws is not None else None,
                                    stream.cuda_stream)
            return out
        stages, final = self._plans_for(elem_bytes, b)
        bufs = [torch.empty_like(src), torch.empty_like(src)]
        cur = src
        with torch.cuda.device(x.device):
            for i, p in enumerate(stages):
                dst = bufs[i & 1]
                B.bmmc_execute_ce(p.handle, cur.data_ptr(), dst.data_ptr(), None, key,
                                  stream.cuda_stream)
                cur = dst
            if final is not None:
                dst = bufs[len(stages) & 1]
                final(cur, out=dst, stream=stream)
                cur = dst
        return cur if cur is not src else src.clone()
