"""The allocation-free float64 solve (spai_pcg_solve_noalloc).

Some callers cannot allocate device memory while they solve (their own
memory manager or a fixed budget owns the device); this entry point keeps its
working memory in the library's static device array instead.  It must give
the same solution as the allocating entry point spai_pcg_solve, on two calls
in a row (the shared scratch keeps the previous call's contents), and reject
sizes beyond its stated maximum.  Collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fsai

pytestmark = pytest.mark.gpu


def csr_of(spai, n, rowptr, colidx, val):
    return spai.CSRMatrix(n, rowptr.contiguous(), colidx.contiguous(), val.to(torch.float64).contiguous())


def setup_fsai(spai, A):
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    _, _, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, spai.PATTERN_UPPER)
    M = spai.precond_from_values(pat, torch.tensor(gv, device="cuda"), spai.F64, eps=0.0)
    return dA, pat, M, 0.0


def setup_gnn(spai, A, v, eps):
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, pat, torch.tensor(v, device="cuda"), torch.tensor(W.gnn_random_weights(v.shape[1]),
                         device="cuda"), d_node=v.shape[1], g_dtype=spai.F64, eps=eps)
    return dA, pat, M, eps


@pytest.mark.parametrize("case", ["fsai_poisson", "gnn_aniso"])
def test_noalloc_matches_allocating_solve_twice(spai_lib, case):
    spai = spai_lib
    if case == "fsai_poisson":
        A = W.poisson2d(64)
        dA, pat, M, eps = setup_fsai(spai, A)
    else:
        A = W.aniso2d(70, 20.0, 0.8)
        dA, pat, M, eps = setup_gnn(spai, A, W.row_average_feature(A), 3.0)
    p = pat.export()
    g, gt = M.export(spai.F64)
    G = csr_of(spai, A.n, p["rowptr"], p["colidx"], g)
    GT = csr_of(spai, A.n, p["t_rowptr"], p["t_colidx"], gt)
    for call in range(2):
        b = torch.tensor(W.rhs_uniform(A.n, 50 + call), device="cuda")
        x_ref = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r_ref = spai.pcg_solve(dA, M, b, x_ref)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = spai.pcg_solve_noalloc(dA, G, GT, eps, b, x)
        assert r_ref["status"] == 0 and r["status"] == 0
        assert r["iters"] == r_ref["iters"]
        xr = x_ref.cpu().numpy()
        assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-8 * np.linalg.norm(xr)
        assert r["true_rel_res"] <= 1e-8


def test_noalloc_rejects_too_large(spai_lib):
    spai = spai_lib
    A = W.poisson2d(363)  # n = 131769 > 131072
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(spai.SpaiError) as ei:
        spai.pcg_solve_noalloc(dA, dA, dA, 0.0, b, x)
    assert ei.value.code == spai.spai.ERR_TOO_LARGE
    with pytest.raises(spai.SpaiError) as ei:
        small = W.poisson2d(8)
        dS = spai.CSRMatrix.from_numpy(small.n, small.rowptr, small.colidx, small.val)
        spai.pcg_solve_noalloc(dS, dS, dS, 0.0, b[:small.n], x[:small.n], precision=spai.PREC_MIXED)
    assert ei.value.code == spai.spai.ERR_INVALID
