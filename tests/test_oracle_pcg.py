"""Pins for the oracle PCG (Algorithm 1, App. A) and the apply of Eq. 2.

Independent references: dense linear algebra (numpy), scipy's CG (a library
routine) for the special cases G = I and G = D^-1/2, finite termination of CG
and the closeness of recurrence and true residuals at replacements.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import workloads as W
from oracle import fsai, pcg


def identity_g(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return np.where(A.colidx == rows, 1.0, 0.0)


def jacobi_g(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.val[A.colidx == rows]
    return np.where(A.colidx == rows, 1.0 / np.sqrt(diag[rows]), 0.0)


def scipy_matrix(A):
    return sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))


def test_apply_matches_dense_formula():
    A = W.random_spd_sparse(30, 0.1, 7)
    g = W.rng(1).standard_normal(A.nnz)
    G = np.zeros((A.n, A.n))
    G[np.repeat(np.arange(A.n), np.diff(A.rowptr)), A.colidx] = g
    r = W.rhs_normal(A.n, 2)
    eps = 0.3
    s = pcg.spai_apply(A.n, A.rowptr, A.colidx, g, eps)(r)
    assert np.allclose(s, (G @ G.T + eps * np.eye(A.n)) @ r, rtol=1e-13, atol=1e-13)
    # Eq. 2 written entry by entry: s_j = eps r_j + sum_l G_jl sum_k G_kl r_k
    j = 5
    manual = eps * r[j] + sum(G[j, l] * sum(G[k, l] * r[k] for k in range(A.n)) for l in range(A.n))
    assert math.isclose(s[j], manual, rel_tol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_solution_matches_dense_solve(seed):
    A = W.random_spd_sparse(40, 0.1, seed)
    b = W.rhs_uniform(A.n, seed + 10)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    res = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-14)
    x = np.linalg.solve(A.to_dense(), b)
    assert res.status == pcg.CONVERGED
    assert np.linalg.norm(res.x - x) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("which", ["identity", "jacobi"])
def test_special_cases_reproduce_scipy_cg(which):
    # G = I (plain CG) and G = D^-1/2 with eps = 0 (Jacobi PCG) against scipy's CG
    A = W.aniso2d(12, 30.0, 0.9)
    b = W.rhs_uniform(A.n, 3)
    g = identity_g(A) if which == "identity" else jacobi_g(A)
    ours = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g, 0.0),
                   rtol=1e-10, replace_period=0, record_x=True)
    xs = []
    if which == "identity":
        M = None
    else:
        diag = A.to_dense().diagonal()
        M = sla.LinearOperator((A.n, A.n), matvec=lambda v: v / diag)
    x, info = sla.cg(scipy_matrix(A), b, rtol=1e-10, atol=0.0, M=M, callback=lambda xk: xs.append(xk.copy()))
    assert info == 0 and ours.status == pcg.CONVERGED
    assert abs(len(xs) - ours.iters) <= 1
    k = min(len(xs), ours.iters)
    xn = np.linalg.norm(x)
    for i in range(k):
        assert np.linalg.norm(xs[i] - ours.x_history[i]) <= 1e-10 * xn, i


def test_finite_termination():
    # CG on a matrix with k distinct eigenvalues terminates in at most k steps
    n = 24
    q, _ = np.linalg.qr(W.rng(11).standard_normal((n, n)))
    lam = np.array([1.0, 2.0, 5.0, 9.0])[np.arange(n) % 4]
    Ad = (q * lam) @ q.T
    Ad = 0.5 * (Ad + Ad.T)
    A = W.dense_to_csr(Ad)
    b = W.rhs_uniform(n, 12)
    res = pcg.pcg(n, A.rowptr, A.colidx, A.val, b,
                  pcg.spai_apply(n, A.rowptr, A.colidx, identity_g(A), 0.0), rtol=1e-10)
    assert res.status == pcg.CONVERGED and res.iters <= 4


def test_recurrence_tracks_true_residual_poisson64():
    A = W.poisson2d(64)
    b = W.rhs_uniform(A.n, W.BASE_SEED + 1)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    res = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-8)
    assert res.status == pcg.CONVERGED
    assert res.true_rel_res <= 1e-8
    bn = np.linalg.norm(b)
    assert len(res.replace_gaps) >= 2
    for i, gap, _ in res.replace_gaps:
        assert gap <= 1e-10 * bn, (i, gap)
    # FSAI beats unpreconditioned CG on this problem
    plain = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b,
                    pcg.spai_apply(A.n, A.rowptr, A.colidx, identity_g(A), 0.0), rtol=1e-8)
    assert res.iters < plain.iters


def test_literal_criterion_agrees_when_m_is_identity():
    A = W.poisson2d(20)
    b = W.rhs_uniform(A.n, 5)
    ap = pcg.spai_apply(A.n, A.rowptr, A.colidx, identity_g(A), 0.0)
    a = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, ap, rtol=1e-8, replace_period=0)
    p = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, ap, rtol=1e-8, replace_period=0, criterion=pcg.PRECOND)
    assert a.status == p.status == pcg.CONVERGED
    assert abs(a.iters - p.iters) <= 1


def test_zero_rhs_and_breakdown():
    A = W.poisson2d(6)
    res = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, np.zeros(A.n), lambda r: r)
    assert res.status == pcg.CONVERGED and res.iters == 0 and not res.x.any()
    # an indefinite "matrix" breaks down with d^T q <= 0
    neg = W.CSR(A.n, A.rowptr, A.colidx, -A.val)
    res = pcg.pcg(A.n, neg.rowptr, neg.colidx, neg.val, W.rhs_uniform(A.n, 1), lambda r: r)
    assert res.status == pcg.BREAKDOWN
