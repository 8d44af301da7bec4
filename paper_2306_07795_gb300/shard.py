"""One BMMC permutation of an array sharded over the ranks of a process group
(include/bmmc_shard.h): local permutations on each rank and all-to-all
exchanges between them.

The array of 2^n elements is split by its top g index bits over 2^g ranks
(rank r holds the elements whose index has top bits r, in order).  The
library plans the steps on the host; each rank runs them on its own shard:
a LOCAL step is a BMMC on the rank's n - g bits (the rank's own complement),
run by the library's kernels; an EXCHANGE is torch.distributed's
all_to_all_single with equal splits (NCCL between GPUs).  The paper relates
BMMCs over several memories to the parallel-disk BMMC algorithms it cites
(Sec. 7).
"""

from . import _binding as B
from .plan import Plan


class ShardedPlan:
    """out[A x + c] = in[x] for an array sharded over 2^g ranks."""

    def __init__(self, n, g, rows, c=0, elem_bytes=4, flags=B.BMMC_PLAN_PAPER):
        self.n, self.g = int(n), int(g)
        self.rows = [int(r) for r in rows]
        self.c = int(c)
        self.elem_bytes = int(elem_bytes)
        self.flags = flags
        self._h = B.bmmc_shard_plan_create(self.n, self.g, self.rows, self.c)
        self._local = {}

    @property
    def num_steps(self):
        return B.bmmc_shard_plan_num_steps(self._h)

    @property
    def num_exchanges(self):
        return sum(1 for i in range(self.num_steps)
                   if B.bmmc_shard_plan_step(self._h, i, 0, self.n - self.g)[0]
                   == B.BMMC_SHARD_EXCHANGE)

    def verify(self):
        return B.bmmc_shard_plan_verify(self._h)

    def steps(self, rank):
        """[(kind, rows, c)] as rank `rank` runs them."""
        nl = self.n - self.g
        return [B.bmmc_shard_plan_step(self._h, i, rank, nl) for i in range(self.num_steps)]

    def _gpu_local(self, step, rank, rows, c, x):
        key = (step, rank)
        plan = self._local.get(key)
        if plan is None:
            plan = self._local[key] = Plan(self.n - self.g, rows, c, self.elem_bytes,
                                           flags=self.flags)
        return plan(x)

    def __call__(self, x, rank, group=None, local=None):
        """Permute this rank's shard x (contiguous, 2^(n-g) elements of
        elem_bytes, any dtype) and return the rank's shard of the result.
        Every rank of `group` (2^g of them) calls this with its own shard.
        local(rows, c, x) runs a LOCAL step; by default the library's kernels
        on x's device."""
        import torch.distributed as dist
        world = dist.get_world_size(group)
        if world != 1 << self.g:
            raise ValueError("the plan needs 2^g = %d ranks, the group has %d"
                             % (1 << self.g, world))
        if x.numel() * x.element_size() != (1 << (self.n - self.g)) * self.elem_bytes:
            raise ValueError("shard holds %d bytes, the plan needs %d"
                             % (x.numel() * x.element_size(),
                                (1 << (self.n - self.g)) * self.elem_bytes))
        shape = x.shape
        x = x.contiguous().view(1 << (self.n - self.g), -1)
        for i, (kind, rows, c) in enumerate(self.steps(rank)):
            if kind == B.BMMC_SHARD_EXCHANGE:
                y = x.new_empty(x.shape)
                dist.all_to_all_single(y, x, group=group)
                x = y
            elif local is not None:
                x = local(rows, c, x)
            else:
                x = self._gpu_local(i, rank, rows, c, x.view(-1)).view(x.shape)
        return x.view(shape)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            try:
                B.bmmc_shard_plan_destroy(h)
            except Exception:
                pass
            self._h = None
