"""Classical factorised sparse approximate inverse (oracle).

The paper builds M^-1 = G G^T + eps I (Eq. 1) and cites the factorised SPAI of
Kolotilina and Yeremin as the classical construction of such a factor.  That
method fixes a lower-triangular pattern and computes, independently for every
row i with row pattern P_i = {j <= i : A_ij != 0} (ascending, i last):

    solve  A[P_i, P_i] y = e_last          (dense, small)
    W[i, P_i] = y / sqrt(y_last)

so that (W A W^T)_ii = 1 and W^T W approximates A^-1.  With the paper's
convention M^-1 = G G^T the factor is G = W^T (upper triangular) and G^T = W.

Pins: A diagonal gives W = D^-1/2; a complete lower pattern on a dense SPD A
gives W = L^-1 from the Cholesky factor A = L L^T, so G G^T = A^-1.
"""
from __future__ import annotations

import numpy as np

from . import pattern as P


def fsai_lower_factor(n: int, rowptr: np.ndarray, colidx: np.ndarray, val: np.ndarray):
    """Return W as CSR on LOWER(A): (rowptr, colidx, wval)."""
    lrp, lci, _ = P.restrict(n, rowptr, colidx, P.LOWER)
    # dense lookup of A entries restricted to a row pattern
    wval = np.empty(lci.shape[0], dtype=np.float64)
    a_rows = [dict(zip(colidx[rowptr[i]:rowptr[i + 1]].tolist(), val[rowptr[i]:rowptr[i + 1]].tolist()))
              for i in range(n)]
    for i in range(n):
        pi = lci[lrp[i]:lrp[i + 1]].tolist()
        k = len(pi)
        sub = np.empty((k, k))
        for a, ja in enumerate(pi):
            row = a_rows[ja]
            for c, jc in enumerate(pi):
                sub[a, c] = row.get(jc, 0.0)
        rhs = np.zeros(k)
        rhs[-1] = 1.0
        chol = np.linalg.cholesky(sub)
        y = np.linalg.solve(chol.T, np.linalg.solve(chol, rhs))
        wval[lrp[i]:lrp[i + 1]] = y / np.sqrt(y[-1])
    return lrp, lci, wval


def fsai_g(n: int, rowptr: np.ndarray, colidx: np.ndarray, val: np.ndarray):
    """G = W^T on UPPER(A), as CSR (rowptr, colidx, gval)."""
    lrp, lci, wval = fsai_lower_factor(n, rowptr, colidx, val)
    urp, uci, perm = P.transpose(n, lrp, lci)
    gval = np.empty_like(wval)
    gval[perm] = wval
    return urp, uci, gval
