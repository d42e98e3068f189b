"""GB300 (sm_103a) implementation of the IBSN hot path for exact discrete OT.

The numerical work runs in the CUDA library built from ``csrc/`` (see
``build.py``) behind the C ABI of ``include/ibsn.h``; ``api`` marshals torch
tensors into it.
"""

from .api import (  # noqa: F401
    COST_DENSE_F32,
    COST_DENSE_F64,
    COST_GRID2D,
    PREC_FP64,
    PREC_MIXED,
    Context,
    Problem,
    alloc_workspace,
    params,
    solve,
    solve_batch,
    workspace_size,
)
from . import warmstart  # noqa: F401,E402
