"""Plan: a BMMC permutation bound to an array shape, callable on CUDA tensors.

A plan is the paper's permutation out[A x + c] = in[x] (Sec. 3) after
validation, classification and factorisation (Sec. 5.1, 5.2) into at most
two tiled passes (Sec. 4), all done on the host by the C library."""

from . import _binding as B


def _current_raw_stream(dev):
    """The cudaStream_t of PyTorch's current stream on `dev`, as an int.  The
    raw accessor skips building a Stream object (about 3 us per call)."""
    import torch
    getter = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    if getter is not None:
        return getter(dev.index)
    return torch.cuda.current_stream(dev).cuda_stream


class Plan:
    """out[A x + c] = in[x] over arrays of 2^n elements of elem_bytes bytes.

    rows: n row masks (bit j of rows[i] is a_ij); c: complement mask.
    flags: BMMC_PLAN_PAPER (one tiled pass, or two after the UL.P
    factorisation) or BMMC_PLAN_SINGLE_PASS.
    """

    def __init__(self, n, rows, c=0, elem_bytes=4, flags=B.BMMC_PLAN_PAPER,
                 seg_bits=0, cta_tile_log2=0, tile_order=0, _handle=None):
        self.n = int(n)
        self.rows = [int(r) for r in rows]
        self.c = int(c)
        self.elem_bytes = int(elem_bytes)
        self.flags = flags
        self.seg_bits = seg_bits
        self.cta_tile_log2 = cta_tile_log2
        self.tile_order = tile_order
        if _handle is not None:
            self._h = _handle
        else:
            self._h = B.bmmc_plan_create_ex(self.n, self.rows, self.c,
                                            self.elem_bytes, flags, seg_bits,
                                            cta_tile_log2, tile_order)
        self._inverse = None
        self._ws_bytes = None

    # -- plan queries -------------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def nbytes(self):
        return (1 << self.n) * self.elem_bytes

    @property
    def num_passes(self):
        return B.bmmc_plan_num_passes(self._h)

    @property
    def workspace_bytes(self):
        return B.bmmc_plan_workspace_bytes(self._h)

    def pass_matrices(self):
        return [B.bmmc_plan_pass_matrix(self._h, self.n, i)
                for i in range(self.num_passes)]

    def describe(self):
        return B.bmmc_plan_describe(self._h)

    def verify(self, max_ctas=0):
        return B.bmmc_plan_verify(self._h, max_ctas)

    def inverse(self):
        """Plan of (A^{-1}, A^{-1} c), cached."""
        if self._inverse is None:
            h = B.bmmc_plan_inverse(self._h)
            inv_rows, inv_c = B.bmmc_plan_matrix(h, self.n)
            self._inverse = Plan(self.n, inv_rows, inv_c, self.elem_bytes,
                                 self.flags, self.seg_bits, self.cta_tile_log2,
                                 self.tile_order, _handle=h)
        return self._inverse

    def lift(self, b):
        """Plan of the same permutation on each of 2^b arrays stored one after
        another (diag(A, I_b), bmmc_plan_lift)."""
        if b == 0:
            return self
        h = B.bmmc_plan_lift(self._h, b)
        rows, c = B.bmmc_plan_matrix(h, self.n + b)
        return Plan(self.n + b, rows, c, self.elem_bytes, self.flags, self.seg_bits,
                    self.cta_tile_log2, self.tile_order, _handle=h)

    # -- execution ----------------------------------------------------------
    def _check_tensor(self, t, name):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor (there is no CPU path)" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() * t.element_size() != self.nbytes:
            raise ValueError("%s holds %d bytes, the plan needs %d"
                             % (name, t.numel() * t.element_size(), self.nbytes))

    def __call__(self, x, out=None, stream=None, workspace=None):
        """Permute tensor x (any dtype; its bytes are 2^n elements of
        elem_bytes).  Returns out (allocated like x if not given)."""
        import torch

        self._check_tensor(x, "x")
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check_tensor(out, "out")
        dev = x.device
        raw = stream.cuda_stream if stream is not None else _current_raw_stream(dev)
        ws_bytes = self._ws_bytes
        if ws_bytes is None:
            ws_bytes = self._ws_bytes = self.workspace_bytes  # plans are immutable
        if ws_bytes and workspace is None:
            workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        ws_ptr = workspace.data_ptr() if ws_bytes else None
        if dev.index == torch.cuda.current_device():
            code = B.lib().bmmc_execute_ws(self._h, x.data_ptr(), out.data_ptr(), ws_ptr, raw)
        else:
            with torch.cuda.device(dev):
                code = B.lib().bmmc_execute_ws(self._h, x.data_ptr(), out.data_ptr(),
                                               ws_ptr, raw)
        if code != B.BMMC_OK:
            raise B.BmmcError(code, "bmmc_execute_ws")
        return out

    def execute_host(self, host_in, host_out, dev_in, dev_out, stream=None, workspace=None):
        """Host tensor host_in -> host tensor host_out through the device
        staging tensors dev_in, dev_out (bmmc_execute_host: upload, the
        plan's passes, download, in order on `stream`).  Asynchronous: read
        host_out after the stream synchronises.  Pinned host tensors make the
        copies overlap the kernels of other streams."""
        import torch

        for t, name in ((host_in, "host_in"), (host_out, "host_out")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("%s must be a contiguous host tensor" % name)
            if t.numel() * t.element_size() != self.nbytes:
                raise ValueError("%s holds %d bytes, the plan needs %d"
                                 % (name, t.numel() * t.element_size(), self.nbytes))
        self._check_tensor(dev_in, "dev_in")
        self._check_tensor(dev_out, "dev_out")
        if stream is None:
            stream = torch.cuda.current_stream(dev_in.device)
        ws_ptr = workspace.data_ptr() if workspace is not None else None
        with torch.cuda.device(dev_in.device):
            code = B.lib().bmmc_execute_host(self._h, host_in.data_ptr(), host_out.data_ptr(),
                                             dev_in.data_ptr(), dev_out.data_ptr(), ws_ptr,
                                             stream.cuda_stream)
        if code != B.BMMC_OK:
            raise B.BmmcError(code, "bmmc_execute_host")
        return host_out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            try:
                B.bmmc_plan_destroy(h)
            except Exception:
                pass
            self._h = None
