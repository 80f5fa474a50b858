"""Pins of the SAI-loss oracle (Sec. 3.3, Eqs. 7-8)."""
import numpy as np
import pytest

import workloads as W
from oracle import fsai, gnn, sai, spectrum


def dense_loss(A, rp, ci, gv, eps):
    a = spectrum.dense_from_csr(A.n, A.rowptr, A.colidx, A.val)
    g = spectrum.dense_from_csr(A.n, rp, ci, gv)
    e = a @ (g @ g.T + eps * np.eye(A.n)) / gnn.matrix_norm(A.val) - np.eye(A.n)
    return e


def test_unit_probes_sum_to_frobenius_norm():
    # with the probes e_1 .. e_n the estimator is exact: sum_j ||E e_j||^2 = ||E||_F^2
    A = W.random_spd_sparse(30, 0.15, 4)
    rp, ci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    gv = gv * 0.7
    losses = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, rp, ci, gv, 0.05, np.eye(A.n))
    e = dense_loss(A, rp, ci, gv, 0.05)
    assert losses.sum() == pytest.approx(np.sum(e * e), rel=1e-12)
    # and each probe's loss is the squared norm of the matching column of E
    assert np.allclose(losses, np.sum(e * e, axis=0), rtol=1e-12)


def test_exact_scaled_inverse_has_zero_loss():
    # A diagonal, G = diag(sqrt(||A|| / a_ii)), eps = 0: A M^-1 / ||A|| = I
    d = np.array([1.0, 4.0, 9.0, 0.25])
    n = d.size
    rp, ci = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    g = np.sqrt(np.mean(d) / d)
    w = W.rhs_normal(n * 3, 5).reshape(n, 3)
    assert np.abs(sai.sai_loss(n, rp, ci, d, rp, ci, g, 0.0, w)).max() < 1e-28


def test_scale_invariance():
    A = W.poisson2d(8)
    rp, ci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    w = W.rhs_normal(A.n * 2, 9).reshape(A.n, 2)
    l1 = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, rp, ci, gv, 0.1, w)
    l2 = sai.sai_loss(A.n, A.rowptr, A.colidx, 37.0 * A.val, rp, ci, gv, 0.1, w)
    assert np.allclose(l1, l2, rtol=1e-12)


def test_gaussian_probes_estimate_frobenius_norm():
    # E_w ||E w||^2 = ||E||_F^2; 4000 probes: the sample mean is within 5 %
    A = W.random_spd_sparse(20, 0.2, 6)
    rp, ci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    w = np.random.default_rng(3).standard_normal((A.n, 4000))
    est = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, rp, ci, gv, 0.2, w).mean()
    e = dense_loss(A, rp, ci, gv, 0.2)
    assert est == pytest.approx(np.sum(e * e), rel=0.05)
