"""Condition numbers of the preconditioned matrix (oracle).

Sec. 4.5 of the paper measures a preconditioner by the spectrum of A M^-1:
    kappa         = max_i lambda_i / min_i lambda_i
    kappa_Kaporin = ((1/N) sum_i lambda_i) / (prod_i lambda_i)^(1/N)
(arithmetic over geometric mean of the eigenvalues).

* ``preconditioned_eigenvalues``: all eigenvalues of M^-1 A with
  M^-1 = G G^T + eps I (Eq. 1), dense, for small n.  M^-1 A is similar to
  C^T A C where M^-1 = C C^T (Cholesky), a symmetric matrix, so its
  eigenvalues are real and positive.
* ``lanczos_tridiagonal``: the tridiagonal matrix T_k that CG builds
  implicitly (the CG / Lanczos relation): with the step lengths alpha_j and
  the ratios beta_j of k PCG iterations,
      T[j, j]   = 1 / alpha_j + beta_{j-1} / alpha_{j-1}   (beta_{-1} = 0)
      T[j, j+1] = sqrt(beta_j) / alpha_j.
  Its eigenvalues (Ritz values) approximate those of M^-1 A from inside, the
  extreme ones first, so max / min of them estimates kappa from a solve's own
  coefficients without any extra matrix work.
"""
from __future__ import annotations

import numpy as np


def dense_from_csr(n, rowptr, colidx, val) -> np.ndarray:
    a = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    np.add.at(a, (rows, np.asarray(colidx, dtype=np.int64)), np.asarray(val, dtype=np.float64))
    return a


def preconditioned_eigenvalues(n, rowptr, colidx, val, g_rowptr, g_colidx, g_val, eps) -> np.ndarray:
    """Ascending eigenvalues of (G G^T + eps I) A."""
    a = dense_from_csr(n, rowptr, colidx, val)
    g = dense_from_csr(n, g_rowptr, g_colidx, g_val)
    minv = g @ g.T + eps * np.eye(n)
    c = np.linalg.cholesky(minv)
    return np.linalg.eigvalsh(c.T @ a @ c)


def kappa(lams) -> float:
    lams = np.asarray(lams, dtype=np.float64)
    return float(lams.max() / lams.min())


def kappa_kaporin(lams) -> float:
    """Arithmetic mean over geometric mean (the geometric mean through logs)."""
    lams = np.asarray(lams, dtype=np.float64)
    return float(lams.mean() / np.exp(np.mean(np.log(lams))))


def lanczos_tridiagonal(alphas, betas) -> np.ndarray:
    """T_k from k step lengths and the k - 1 ratios that followed them."""
    alphas = np.asarray(alphas, dtype=np.float64)
    k = alphas.shape[0]
    betas = np.asarray(betas, dtype=np.float64)[: max(k - 1, 0)]
    t = np.zeros((k, k))
    for j in range(k):
        t[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            t[j, j + 1] = t[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return t


def ritz_values(alphas, betas) -> np.ndarray:
    return np.linalg.eigvalsh(lanczos_tridiagonal(alphas, betas))
