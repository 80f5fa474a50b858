"""Pins for the oracle's classical factorised SPAI (the Kolotilina-Yeremin
construction the paper cites beside Eq. 1).  Closed forms: unit diagonal of
W A W^T, Jacobi on diagonal A, exact inverse Cholesky factor on a full
pattern, SPD-ness of G G^T."""
import numpy as np
import pytest

import workloads as W
from oracle import fsai, pcg, pattern as P


def dense_of(n, rp, ci, v):
    d = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    d[rows, ci] = v
    return d


@pytest.mark.parametrize("make", [lambda: W.poisson2d(8), lambda: W.random_spd_sparse(60, 0.08, 5),
                                  lambda: W.aniso2d(7, 50.0, 0.4)])
def test_unit_diagonal_of_w_a_wt(make):
    A = make()
    lrp, lci, wv = fsai.fsai_lower_factor(A.n, A.rowptr, A.colidx, A.val)
    Wd = dense_of(A.n, lrp, lci, wv)
    Ad = A.to_dense()
    diag = np.diag(Wd @ Ad @ Wd.T)
    assert np.max(np.abs(diag - 1.0)) < 1e-13
    assert np.all(np.diag(Wd) > 0)
    # G = W^T on the upper pattern, and G G^T = W^T W is SPD
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    Gd = dense_of(A.n, urp, uci, gv)
    assert np.allclose(Gd, Wd.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(Gd @ Gd.T).min() > 0


def test_diagonal_matrix_gives_jacobi():
    n = 9
    d = np.linspace(0.5, 7.0, n)
    A = W.dense_to_csr(np.diag(d))
    lrp, lci, wv = fsai.fsai_lower_factor(A.n, A.rowptr, A.colidx, A.val)
    assert np.allclose(wv, 1.0 / np.sqrt(d), rtol=1e-15)


def test_diagonal_only_pattern_reproduces_jacobi():
    # restricting a non-diagonal matrix to its diagonal gives D^{-1/2}
    A = W.poisson2d(5)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    keep = A.colidx == rows
    D = W.coo_to_csr(A.n, rows[keep], A.colidx[keep], A.val[keep])
    _, _, wv = fsai.fsai_lower_factor(D.n, D.rowptr, D.colidx, D.val)
    assert np.allclose(wv, 0.5, rtol=1e-15)


def test_full_lower_pattern_is_inverse_cholesky():
    n = 12
    Ad = W.random_dense_spd(n, seed=3, cond=50.0)
    A = W.dense_to_csr(Ad)
    lrp, lci, wv = fsai.fsai_lower_factor(A.n, A.rowptr, A.colidx, A.val)
    Wd = dense_of(n, lrp, lci, wv)
    L = np.linalg.cholesky(Ad)
    assert np.allclose(Wd, np.linalg.inv(L), rtol=1e-10, atol=1e-12)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    Gd = dense_of(n, urp, uci, gv)
    assert np.allclose(Gd @ Gd.T, np.linalg.inv(Ad), rtol=1e-9, atol=1e-11)
    # PCG with M^-1 = A^-1 converges in one iteration
    b = W.rhs_uniform(n, 4)
    res = pcg.pcg(n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(n, urp, uci, gv, 0.0), rtol=1e-10)
    assert res.status == pcg.CONVERGED and res.iters == 1


def test_poisson64_counts():
    A = W.poisson2d(64)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    assert urp[-1] == 12160
    rows = np.repeat(np.arange(A.n), np.diff(urp))
    assert np.all(uci >= rows)
    assert P.validate_csr(A.n, A.rowptr, A.colidx) is None
