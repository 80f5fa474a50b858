"""Preconditioned CG with the factorised SPAI preconditioner (oracle).

* ``spmv``: y = A x for CSR A, each row summed in stored order.
* ``spai_apply``: s = M^-1 r with M^-1 = G G^T + eps I (Eq. 1), computed as in
  Eq. 2:  s_j = eps r_j + sum_l G_jl (sum_k G_kl r_k).  The inner sum is G^T r
  formed by scattering each entry G_kl r_k into position l (the definition of
  a transposed product; no explicit transpose is built here).
* ``pcg``: Algorithm 1 (App. A), the standard PCG template with the true
  residual r = b - A x recomputed every 50 iterations.

Reading of Algorithm 1 (the paper prints s, delta, beta and the d update
inside the else-branch of the replacement test, which would leave d stale on
every replacement iteration; the template it cites updates them every
iteration): only the r update is conditional,
    if i % period == 0:  r = b - A x   else:  r = r - alpha q
and the apply, delta, beta and d = s + beta d happen every iteration.

Stopping (the paper's tables stop on ||b - A x|| / ||b|| < rtol, Sec. 4.2;
Algorithm 1 tests delta_new <= tol^2 delta_0):
* criterion "residual" (default): after the r update, if ||r|| <= rtol ||b||
  the true residual b - A x replaces r and is tested again; the solve ends
  only if the true residual passes, else it continues from the replaced r;
* criterion "precond": Algorithm 1's own test on delta.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RESIDUAL, PRECOND = 0, 1
CONVERGED, NOT_CONVERGED, BREAKDOWN = 0, 1, 2


def spmv(n, rowptr, colidx, val, x):
    """y_i = sum over stored entries of row i of A_ij x_j (in stored order)."""
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    prod = np.asarray(val, dtype=np.float64) * np.asarray(x, dtype=np.float64)[colidx]
    return np.bincount(rows, weights=prod, minlength=n)


def spmv_transpose(n, rowptr, colidx, val, r):
    """t_l = sum_k A_kl r_k  (the product with the transpose, by scatter)."""
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    prod = np.asarray(val, dtype=np.float64) * np.asarray(r, dtype=np.float64)[rows]
    return np.bincount(np.asarray(colidx, dtype=np.int64), weights=prod, minlength=n)


def spai_apply(n, g_rowptr, g_colidx, g_val, eps):
    """Return r -> G (G^T r) + eps r  (Eq. 1 applied as in Eq. 2)."""
    def apply(r):
        t = spmv_transpose(n, g_rowptr, g_colidx, g_val, r)
        return spmv(n, g_rowptr, g_colidx, g_val, t) + eps * np.asarray(r, dtype=np.float64)
    return apply


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    status: int
    history: list          # ||r|| after each iteration, history[0] = ||r_0||
    true_rel_res: float
    alphas: list
    betas: list
    x_history: list | None = None     # x after each iteration (record_x=True)
    replace_gaps: list | None = None  # (i, ||r_rec - r_true||, ||r_true||) at replacements


def pcg(n, rowptr, colidx, val, b, apply_minv, x0=None, rtol=1e-8, max_iter=None,
        replace_period=50, criterion=RESIDUAL, record_x=False) -> PCGResult:
    """Algorithm 1 with the reading stated in the module docstring."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if max_iter is None:
        max_iter = min(10 * n, 10 ** 6)
    A = lambda v: spmv(n, rowptr, colidx, val, v)  # noqa: E731
    bb = float(b @ b)
    tol2 = rtol * rtol * bb
    alphas, betas = [], []
    if bb == 0.0:
        return PCGResult(np.zeros(n), 0, CONVERGED, [0.0], 0.0, alphas, betas)

    r = b - A(x)
    rr = float(r @ r)
    hist = [math.sqrt(rr)]
    if criterion == RESIDUAL and rr <= tol2:
        return PCGResult(x, 0, CONVERGED, hist, math.sqrt(rr / bb), alphas, betas)
    s = apply_minv(r)
    d = s.copy()
    delta = float(r @ s)
    delta0 = delta
    status = NOT_CONVERGED
    xs = [] if record_x else None
    gaps = []
    i = 0
    while i < max_iter:
        if criterion == PRECOND and not delta > rtol * rtol * delta0:
            status = CONVERGED
            break
        q = A(d)
        dq = float(d @ q)
        if not (dq > 0.0) or not math.isfinite(dq):
            status = BREAKDOWN
            break
        alpha = delta / dq
        alphas.append(alpha)
        x = x + alpha * d
        if replace_period and i % replace_period == 0:
            r_rec = r - alpha * q
            r = b - A(x)
            gaps.append((i, float(np.linalg.norm(r_rec - r)), float(np.linalg.norm(r))))
        else:
            r = r - alpha * q
        rr = float(r @ r)
        i += 1
        if record_x:
            xs.append(x.copy())
        if criterion == RESIDUAL and rr <= tol2:
            r = b - A(x)                 # confirm with the true residual
            rr = float(r @ r)
            hist.append(math.sqrt(rr))
            if rr <= tol2:
                status = CONVERGED
                break
        else:
            hist.append(math.sqrt(rr))
        s = apply_minv(r)
        delta_old = delta
        delta = float(r @ s)
        if not (delta > 0.0) or not math.isfinite(delta):
            if criterion == PRECOND and delta == 0.0:
                status = CONVERGED
            else:
                status = BREAKDOWN
            break
        beta = delta / delta_old
        betas.append(beta)
        d = s + beta * d
    res = b - A(x)
    return PCGResult(x, i, status, hist, math.sqrt(float(res @ res) / bb), alphas, betas, xs, gaps)


def true_rel_residual(n, rowptr, colidx, val, x, b) -> float:
    """||b - A x|| / ||b|| in float64."""
    b = np.asarray(b, dtype=np.float64)
    r = b - spmv(n, rowptr, colidx, val, x)
    return math.sqrt(float(r @ r) / float(b @ b))
