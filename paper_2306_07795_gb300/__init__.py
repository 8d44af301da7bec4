"""BMMC permutations on GB300 (sm_103a).

A BMMC permutation of an array of 2^n elements sends the element at index x
to index A x + c over F2 (Bouverot-Dupuis & Sheeran, Sec. 3).  The work runs
in hand-written CUDA kernels behind the C ABI of ``include/bmmc.h``; this
package is a thin binding over it, with PyTorch supplying device memory and
streams.

    plan = Plan(n, rows, c, elem_bytes=4)
    y = plan(x)            # x: contiguous CUDA tensor of 2^n * 4 bytes

There is no CPU path: without the built library and a GPU, execution raises.
"""

from ._binding import (  # noqa: F401
    BMMC_ERR_ALIAS, BMMC_ERR_ALIGN, BMMC_ERR_CUDA, BMMC_ERR_INVALID,
    BMMC_ERR_OOM, BMMC_ERR_SINGULAR, BMMC_ERR_TOO_LARGE, BMMC_ERR_UNSUPPORTED,
    BMMC_OK, BMMC_STATIC_SCRATCH_BYTES, bmmc_execute_static_ws,
    BMMC_PLAN_PAPER, BMMC_PLAN_SINGLE_PASS, BmmcError, bmmc_execute,
    bmmc_execute_ws, bmmc_plan_create, bmmc_plan_create_ex,
    bmmc_plan_describe, bmmc_plan_destroy, bmmc_plan_inverse, bmmc_plan_matrix,
    bmmc_plan_num_passes, bmmc_plan_pass_matrix, bmmc_plan_verify,
    bmmc_plan_workspace_bytes, bmmc_strerror, lib, library_path,
    bmmc_plan_compose, bmmc_parm_matrix,
)
from .plan import Plan  # noqa: F401
