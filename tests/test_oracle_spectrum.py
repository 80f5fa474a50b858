"""Pins of the condition-number oracle (Sec. 4.5) against closed forms and
brute force."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fsai, pcg, spectrum


def identity_csr(n):
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n)


def test_diagonal_closed_forms():
    # A = diag(d), G = I, eps = 0: the eigenvalues are d
    d = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    n = d.size
    rp, ci, one = identity_csr(n)
    lam = spectrum.preconditioned_eigenvalues(n, rp, ci, d, rp, ci, one, 0.0)
    assert np.allclose(lam, d, rtol=1e-14)
    assert spectrum.kappa(lam) == pytest.approx(16.0, rel=1e-14)
    # mean 6.2, geometric mean (2^10)^(1/5) = 4
    assert spectrum.kappa_kaporin(lam) == pytest.approx(6.2 / 4.0, rel=1e-14)
    # G = c I, eps = e: eigenvalues (c^2 + e) d
    lam2 = spectrum.preconditioned_eigenvalues(n, rp, ci, d, rp, ci, 3.0 * one, 0.5)
    assert np.allclose(lam2, 9.5 * d, rtol=1e-14)


def test_kaporin_is_one_iff_equal_and_exceeds_one_otherwise():
    assert spectrum.kappa_kaporin([2.0, 2.0, 2.0]) == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(5):
        lam = rng.uniform(0.1, 10.0, size=20)
        k = spectrum.kappa_kaporin(lam)
        assert k > 1.0 and k <= spectrum.kappa(lam)   # AM/GM <= max/min


def test_exact_fsai_of_dense_spd_gives_identity_spectrum():
    # a full lower pattern on a dense SPD matrix makes G G^T = A^-1
    a = W.random_dense_spd(12, seed=5, cond=50.0)
    A = W.dense_to_csr(a)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    lam = spectrum.preconditioned_eigenvalues(A.n, A.rowptr, A.colidx, A.val, urp, uci, gv, 0.0)
    assert np.allclose(lam, 1.0, atol=1e-10)


def test_ritz_values_of_cg_on_distinct_spectrum():
    # CG on a matrix with 5 distinct eigenvalues ends in 5 steps, and T_5 has
    # exactly those eigenvalues (the CG / Lanczos relation)
    vals = np.array([1.0, 3.0, 7.0, 20.0, 50.0])
    d = np.repeat(vals, 8)
    n = d.size
    rp, ci, _ = identity_csr(n)
    b = W.rhs_uniform(n, 7)
    res = pcg.pcg(n, rp, ci, d, b, lambda r: r.copy(), rtol=1e-13, replace_period=0)
    assert len(res.alphas) >= 5          # 5 in exact arithmetic (a 6th may follow rounding)
    assert res.history[5] <= 1e-10 * res.history[0]
    ritz = spectrum.ritz_values(res.alphas[:5], res.betas[:4])
    assert np.allclose(ritz, vals, rtol=1e-9)


def test_ritz_kappa_matches_dense_after_convergence():
    # Poisson 2D with the FSAI factor: extreme Ritz values of a converged solve
    # reproduce the dense extreme eigenvalues of M^-1 A
    A = W.poisson2d(12)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    lam = spectrum.preconditioned_eigenvalues(A.n, A.rowptr, A.colidx, A.val, urp, uci, gv, 0.0)
    b = W.rhs_uniform(A.n, 11)
    res = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-12,
                  replace_period=0)
    ritz = spectrum.ritz_values(res.alphas, res.betas[: len(res.alphas) - 1])
    # Ritz values lie inside the spectrum and the extreme ones converge first
    assert ritz.max() <= lam.max() * (1 + 1e-12) and ritz.min() >= lam.min() * (1 - 1e-12)
    assert ritz.max() == pytest.approx(lam.max(), rel=1e-3)
    assert ritz.min() == pytest.approx(lam.min(), rel=1e-3)
    assert math.isclose(spectrum.kappa(ritz), spectrum.kappa(lam), rel_tol=2e-3)
