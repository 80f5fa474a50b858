"""SAI loss of a preconditioner (oracle).

Sec. 3.3 of the paper trains G with the scale-invariant aligned-identity
loss, estimated with random probe vectors w (Hutchinson's estimator of the
Frobenius norm, Eq. 7):

    L_SAI(A, M^-1, w) = || (A M^-1 w) / ||A|| - w ||_2^2,

with ||A|| = mean |A_ij| over stored entries and M^-1 = G G^T + eps I
(Eq. 1).  Its expectation over w ~ N(0, I) is ||A M^-1 / ||A|| - I||_F^2
(Eq. 8).  Only the forward value is computed here.
"""
from __future__ import annotations

import numpy as np

from . import gnn, pcg


def sai_loss(n, rowptr, colidx, val, g_rowptr, g_colidx, g_val, eps, w) -> np.ndarray:
    """Loss of every probe: w is (n, k); returns k values."""
    w = np.asarray(w, dtype=np.float64).reshape(n, -1)
    apply = pcg.spai_apply(n, g_rowptr, g_colidx, g_val, eps)
    nrm = gnn.matrix_norm(val)
    out = np.empty(w.shape[1])
    for j in range(w.shape[1]):
        v = apply(w[:, j])                       # M^-1 w
        u = pcg.spmv(n, rowptr, colidx, val, v)  # A M^-1 w
        e = u / nrm - w[:, j]
        out[j] = float(e @ e)
    return out
