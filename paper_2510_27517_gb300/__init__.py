"""GB300-native SPAI-preconditioned conjugate gradients with a GNN-built factor.

M^-1 = G G^T + eps I (Eq. 1 of the paper), G on A's sparsity pattern, filled by
the GNN forward pass of Sec. 3.2.2; PCG is Algorithm 1 (App. A).  All compute
runs in the CUDA library libspai.so (C ABI: include/spai.h); this package is
its Python binding.
"""
from .spai import (  # noqa: F401
    BF16, CRIT_PRECOND, CRIT_RESIDUAL, F16, F32, F64, MSG_LATENT, MSG_RAW, PATTERN_FULL, PATTERN_LOWER,
    PATTERN_UPPER, PREC_F64, PREC_MIXED, CSRMatrix, adamw_step, Pattern, Precond, Server, SpaiError, System, build_pattern,
    gnn_grad, gnn_precond, kernel_launches, lib, pcg_solve, pcg_solve_batched, pcg_solve_noalloc, pcg_solve_host, precond_from_values,
    ritz_extremes, ritz_kaporin, sai_loss, sai_loss_grad, selftest_wait_timeout, system_create, system_solve,
)
