"""BMMC permutations on GB300 (sm_103a).

A BMMC permutation of an array of 2^n elements sends the element at index x
to index A x + c over F2 (Bouverot-Dupuis & Sheeran, Sec. 3).  The work runs
in hand-written CUDA kernels behind the C ABI of ``include/*.h``; this
package is a thin binding over it, with PyTorch supplying device memory and
streams.

    plan = Plan(n, rows, c, elem_bytes=4)
    y = plan(x)            # x: contiguous CUDA tensor of 2^n * 4 bytes

Every C entry point is available here under its own name (bmmc_*), with the
status codes and flags (BMMC_*).  There is no CPU path: without the built
library and a GPU, execution raises.
"""

from . import _binding
from ._binding import BmmcError, lib, library_path  # noqa: F401
from .plan import Plan  # noqa: F401

for _name in dir(_binding):
    if _name.startswith(("bmmc_", "BMMC_")):
        globals()[_name] = getattr(_binding, _name)
del _name
