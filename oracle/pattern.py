"""Sparsity pattern of G and its explicit transpose (oracle).

Sec. 3.2.2 (after Eq. 5): the learned G is assembled by putting each G_ij where
A has an entry, keeping A's sparsity pattern exactly (the conclusion repeats
that G's pattern is forced to equal A's).  That is the FULL pattern.

The classical factorised SPAI used as a preconditioner check (Kolotilina and
Yeremin, cited in Sec. 2 and beside Eq. 1) needs a triangular factor.  With
M^-1 = G G^T, G must be *upper* triangular: if A = L L^T then G = L^-T gives
G G^T = A^-1 exactly.  Its transpose G^T = W is lower triangular and is the
factor computed row by row.  Hence both LOWER and UPPER restrictions exist.

The transpose is defined by a counting sort over columns taken in row-major
order, which yields sorted columns in every transposed row.  ``perm[e]`` is the
position, in the transposed arrays, of the entry that original entry ``e``
becomes, so ``val_T[perm[e]] == val[e]``.  For a FULL (symmetric) pattern the
transposed arrays equal the original ones and ``perm[e]`` is the index of the
mirror entry (j, i), an involution.
"""
from __future__ import annotations

import numpy as np

FULL, LOWER, UPPER = 0, 1, 2


def row_of_entry(n: int, rowptr: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr.astype(np.int64)))


def restrict(n: int, rowptr: np.ndarray, colidx: np.ndarray, kind: int):
    """Pattern of G for the given kind: FULL keeps every entry of A,
    LOWER keeps j <= i, UPPER keeps j >= i.  Returns (rowptr, colidx, src)
    where src[e] is the index in A of G's entry e."""
    rows = row_of_entry(n, rowptr)
    cols = colidx.astype(np.int64)
    if kind == FULL:
        keep = np.ones(cols.shape, dtype=bool)
    elif kind == LOWER:
        keep = cols <= rows
    elif kind == UPPER:
        keep = cols >= rows
    else:
        raise ValueError("unknown pattern kind")
    src = np.nonzero(keep)[0]
    counts = np.bincount(rows[keep], minlength=n)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp.astype(np.int32), colidx[keep].astype(np.int32), src.astype(np.int64)


def transpose(n: int, rowptr: np.ndarray, colidx: np.ndarray):
    """Transposed CSR by counting sort.

    Entries are visited in row-major order and appended to the bucket of
    their column, so every transposed row lists its columns (the original
    rows) in ascending order.  Returns (t_rowptr, t_colidx, perm)."""
    nnz = colidx.shape[0]
    rows = row_of_entry(n, rowptr)
    counts = np.bincount(colidx.astype(np.int64), minlength=n)
    t_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=t_rowptr[1:])
    fill = t_rowptr[:-1].copy()
    t_colidx = np.empty(nnz, dtype=np.int64)
    perm = np.empty(nnz, dtype=np.int64)
    for e in range(nnz):  # plain counting sort, one entry at a time
        c = colidx[e]
        p = fill[c]
        fill[c] += 1
        t_colidx[p] = rows[e]
        perm[e] = p
    return t_rowptr.astype(np.int32), t_colidx.astype(np.int32), perm.astype(np.int32)


def transpose_fast(n: int, rowptr: np.ndarray, colidx: np.ndarray):
    """Same result as ``transpose`` via a stable argsort on the column; used
    for inputs too large for the entry-by-entry loop."""
    rows = row_of_entry(n, rowptr)
    order = np.argsort(colidx.astype(np.int64), kind="stable")
    counts = np.bincount(colidx.astype(np.int64), minlength=n)
    t_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=t_rowptr[1:])
    t_colidx = rows[order]
    perm = np.empty(colidx.shape[0], dtype=np.int64)
    perm[order] = np.arange(colidx.shape[0])
    return t_rowptr.astype(np.int32), t_colidx.astype(np.int32), perm.astype(np.int32)


def is_symmetric_pattern(n: int, rowptr: np.ndarray, colidx: np.ndarray) -> bool:
    t_rp, t_ci, _ = transpose_fast(n, rowptr, colidx)
    return bool(np.array_equal(t_rp, rowptr) and np.array_equal(t_ci, colidx))


def validate_csr(n: int, rowptr: np.ndarray, colidx: np.ndarray) -> str | None:
    """Reason the CSR is unusable, or None.  Requirements: rowptr starts at 0
    and never decreases, columns in range, strictly ascending in each row,
    diagonal present in every row."""
    if rowptr.shape[0] != n + 1 or rowptr[0] != 0:
        return "rowptr shape or start"
    if np.any(np.diff(rowptr.astype(np.int64)) < 0):
        return "rowptr decreasing"
    if rowptr[-1] != colidx.shape[0]:
        return "rowptr end != nnz"
    if colidx.size and (colidx.min() < 0 or colidx.max() >= n):
        return "column out of range"
    rows = row_of_entry(n, rowptr)
    same_row = rows[1:] == rows[:-1]
    if np.any(same_row & (colidx[1:] <= colidx[:-1])):
        return "columns not strictly ascending"
    diag = np.zeros(n, dtype=bool)
    diag[rows[colidx == rows]] = True
    if not diag.all():
        return "missing diagonal"
    return None
