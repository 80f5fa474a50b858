"""Pins for the oracle's pattern and transpose (Sec. 3.2.2: G keeps A's pattern).

Checked against brute force on dense boolean matrices, involution properties
and counting identities, so that a wrong index, a dropped entry or an
unsorted row fails here.
"""
import numpy as np
import pytest

import workloads as W
from oracle import pattern as P


def random_pattern(n, density, seed, symmetric=False):
    g = W.rng(seed)
    m = g.random((n, n)) < density
    if symmetric:
        m = m | m.T
    np.fill_diagonal(m, True)
    r, c = np.nonzero(m)
    A = W.coo_to_csr(n, r, c, g.standard_normal(r.size))
    return A, m


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n", [1, 2, 5, 11])
def test_transpose_matches_dense_boolean(seed, n):
    A, m = random_pattern(n, 0.35, seed)
    trp, tci, perm = P.transpose(n, A.rowptr, A.colidx)
    # dense rebuild of the transpose pattern
    t = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(trp))
    t[rows, tci] = True
    assert np.array_equal(t, m.T)
    # columns sorted inside every transposed row
    for i in range(n):
        seg = tci[trp[i]:trp[i + 1]]
        assert np.all(np.diff(seg) > 0)
    # perm maps entry (i,j) to the slot holding (j,i) in the transpose
    arows = np.repeat(np.arange(n), np.diff(A.rowptr))
    for e in range(A.nnz):
        p = perm[e]
        assert tci[p] == arows[e]
        assert trp[A.colidx[e]] <= p < trp[A.colidx[e] + 1]
    assert sorted(perm.tolist()) == list(range(A.nnz))


@pytest.mark.parametrize("seed", range(4))
def test_transpose_twice_is_identity(seed):
    n = 17
    A, _ = random_pattern(n, 0.2, seed)
    trp, tci, perm1 = P.transpose(n, A.rowptr, A.colidx)
    rp2, ci2, perm2 = P.transpose(n, trp, tci)
    assert np.array_equal(rp2, A.rowptr) and np.array_equal(ci2, A.colidx)
    assert np.array_equal(perm2[perm1], np.arange(A.nnz))


@pytest.mark.parametrize("seed", range(4))
def test_full_symmetric_perm_is_involution(seed):
    n = 23
    A, m = random_pattern(n, 0.15, seed, symmetric=True)
    trp, tci, perm = P.transpose(n, A.rowptr, A.colidx)
    assert np.array_equal(trp, A.rowptr) and np.array_equal(tci, A.colidx)
    assert np.array_equal(perm[perm], np.arange(A.nnz))
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    # perm[e] is the mirror entry (j, i)
    assert np.array_equal(rows[perm], A.colidx) and np.array_equal(A.colidx[perm], rows)
    assert P.is_symmetric_pattern(n, A.rowptr, A.colidx)


def test_fast_transpose_equals_counting_sort():
    n = 40
    A, _ = random_pattern(n, 0.2, 99)
    a = P.transpose(n, A.rowptr, A.colidx)
    b = P.transpose_fast(n, A.rowptr, A.colidx)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_lower_upper_counts_and_content():
    A = W.poisson2d(64)
    lrp, lci, lsrc = P.restrict(A.n, A.rowptr, A.colidx, P.LOWER)
    urp, uci, usrc = P.restrict(A.n, A.rowptr, A.colidx, P.UPPER)
    # symmetric pattern with full diagonal: nnz_lower = nnz_upper = (nnz + n) / 2
    assert lci.size == urp[-1] == (A.nnz + A.n) // 2 == 12160
    rows = np.repeat(np.arange(A.n), np.diff(lrp))
    assert np.all(lci <= rows)
    rows_u = np.repeat(np.arange(A.n), np.diff(urp))
    assert np.all(uci >= rows_u)
    # the upper pattern is the transpose of the lower one
    trp, tci, _ = P.transpose(A.n, lrp, lci)
    assert np.array_equal(trp, urp) and np.array_equal(tci, uci)
    frp, fci, fsrc = P.restrict(A.n, A.rowptr, A.colidx, P.FULL)
    assert np.array_equal(frp, A.rowptr) and np.array_equal(fci, A.colidx)
    assert np.array_equal(fsrc, np.arange(A.nnz))


def test_validate_csr_rejects_each_defect():
    A = W.poisson2d(4)
    n = A.n
    assert P.validate_csr(n, A.rowptr, A.colidx) is None
    ci = A.colidx.copy(); ci[1], ci[2] = ci[2], ci[1]
    assert "ascending" in P.validate_csr(n, A.rowptr, ci)
    ci = A.colidx.copy(); ci[0] = n
    assert "range" in P.validate_csr(n, A.rowptr, ci)
    # drop the diagonal of row 0 (first entry of row 0 is the diagonal)
    rp = A.rowptr.copy(); rp[1:] -= 1
    assert P.validate_csr(n, rp, A.colidx[1:]) == "missing diagonal"
    rp = A.rowptr.copy(); rp[2] = rp[1] - 1
    assert "decreasing" in P.validate_csr(n, rp, A.colidx)
