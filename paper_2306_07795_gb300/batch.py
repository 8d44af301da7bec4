"""Batch: many BMMC permutations, one persistent launch per phase.

    b = Batch(plans, ins, outs)     # binds buffers; uploads tables on a stream
    b()                             # launches on the current stream
    g = b.capture()                 # a torch.cuda.CUDAGraph of those launches
    g.replay()

The tables and the two-pass workspace come from PyTorch's allocator and live
as long as the Batch object; the library itself allocates nothing for a batch.
Every array goes through the same passes as alone (Sec. 5.1 / 5.2); batching
is this library's answer to the paper's remark that arrays under 2^20
elements cannot fill a GPU (Sec. 6).
"""

from . import _binding as B


class Batch:
    def __init__(self, plans, ins, outs, workspace=None, stream=None):
        import torch

        if not (len(plans) == len(ins) == len(outs)) or not plans:
            raise ValueError("plans, ins and outs must be non-empty and of equal length")
        self.plans = list(plans)
        self.ins = list(ins)
        self.outs = list(outs)
        for p, x, y in zip(self.plans, self.ins, self.outs):
            p._check_tensor(x, "input")
            p._check_tensor(y, "output")
        dev = self.ins[0].device
        self.device = dev
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        handles = [p.handle for p in self.plans]
        need = B.bmmc_batch_workspace_bytes(handles)
        if need and workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=dev)
        if need and workspace.numel() * workspace.element_size() < need:
            raise ValueError("workspace holds fewer than %d bytes" % need)
        self.workspace = workspace
        self.table = torch.empty(B.bmmc_batch_table_bytes(handles), dtype=torch.uint8,
                                 device=dev)
        # the allocator must not hand these bytes out again before `stream`
        # is done with them
        self.table.record_stream(stream)
        if need:
            workspace.record_stream(stream)
        with torch.cuda.device(dev):
            self._h = B.bmmc_batch_create(
                handles, [x.data_ptr() for x in self.ins],
                [y.data_ptr() for y in self.outs],
                workspace.data_ptr() if need else None, self.table.data_ptr(),
                stream.cuda_stream)

    @property
    def num_launches(self):
        return B.bmmc_batch_num_launches(self._h)

    def describe(self):
        return B.bmmc_batch_describe(self._h)

    @property
    def bytes_moved(self):
        """2 * N * e summed over the arrays (the effective-bandwidth numerator)."""
        return self.describe()["bytes_moved"]

    def __call__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        if stream is not self.stream and stream.cuda_stream != self.stream.cuda_stream:
            stream.wait_stream(self.stream)  # after the table upload
        with torch.cuda.device(self.device):
            B.bmmc_batch_execute(self._h, stream.cuda_stream)

    def capture(self):
        """Record this batch's launches into a CUDA graph and return it."""
        import torch
        self()  # one execution outside capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.device(self.device):
            with torch.cuda.graph(g):
                B.bmmc_batch_execute(self._h, torch.cuda.current_stream(self.device).cuda_stream)
        return g

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            try:
                B.bmmc_batch_destroy(h)
            except Exception:
                pass
            self._h = None
