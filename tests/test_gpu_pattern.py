"""build_pattern on the GPU against the oracle: bit-exact G / G^T patterns and
perm (Sec. 3.2.2: G keeps A's pattern), and rejection of malformed CSR."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pattern as P

pytestmark = pytest.mark.gpu


def cases():
    return {
        "poisson64": W.poisson2d(64),
        "aniso": W.aniso2d(37, 200.0, 1.1),
        "graph": W.graph_laplacian(3000, 24000, seed=5),
        "random": W.random_spd_sparse(500, 0.02, 3),
        "dense_row": dense_row_case(),
        "one": W.dense_to_csr(np.array([[2.0]])),
    }


def dense_row_case():
    # an arrow matrix: row/column 0 couples to everything (a row longer than a tile)
    n = 6000
    rows = np.concatenate([np.zeros(n - 1, int), np.arange(1, n), np.arange(n)])
    cols = np.concatenate([np.arange(1, n), np.zeros(n - 1, int), np.arange(n)])
    vals = np.concatenate([-np.ones(n - 1) * 0.1, -np.ones(n - 1) * 0.1, np.full(n, 1.0)])
    vals[-n] = 0.1 * n + 1.0
    return W.coo_to_csr(n, rows, cols, vals)


@pytest.mark.parametrize("name", list(cases()))
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_pattern_bit_exact(spai_lib, name, kind):
    spai = spai_lib
    A = cases()[name]
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, kind)
    out = {k: v.cpu().numpy() for k, v in pat.export().items()}
    rp, ci, _ = P.restrict(A.n, A.rowptr, A.colidx, kind)
    trp, tci, perm = P.transpose_fast(A.n, rp, ci)
    assert np.array_equal(out["rowptr"], rp)
    assert np.array_equal(out["colidx"], ci)
    assert np.array_equal(out["t_rowptr"], trp)
    assert np.array_equal(out["t_colidx"], tci)
    assert np.array_equal(out["perm"], perm)


def test_pattern_full_equals_counting_sort_oracle(spai_lib):
    spai = spai_lib
    A = W.poisson2d(20)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    out = {k: v.cpu().numpy() for k, v in spai.build_pattern(dA, 0).export().items()}
    trp, tci, perm = P.transpose(A.n, A.rowptr, A.colidx)
    assert np.array_equal(out["perm"], perm) and np.array_equal(out["t_colidx"], tci)


@pytest.mark.parametrize("defect", ["unsorted", "missing_diag", "asym", "col_range", "rowptr"])
def test_bad_csr_rejected(spai_lib, defect):
    spai = spai_lib
    A = W.poisson2d(6)
    rp, ci, v = A.rowptr.copy(), A.colidx.copy(), A.val.copy()
    if defect == "unsorted":
        ci[1], ci[2] = ci[2], ci[1]
    elif defect == "missing_diag":
        # replace row 0's diagonal column by a column not otherwise present in row 0
        ci[0] = 7
        ci[:rp[1]] = np.sort(ci[:rp[1]])
    elif defect == "asym":
        # drop one off-diagonal entry of the last row only
        last = rp[-2]
        keep = np.ones(ci.size, bool)
        keep[last] = False
        ci, v = ci[keep], v[keep]
        rp = rp.copy(); rp[-1] -= 1
    elif defect == "col_range":
        ci[3] = A.n + 5
    elif defect == "rowptr":
        rp = rp.copy(); rp[3], rp[4] = rp[4], rp[3]
    dA = spai.CSRMatrix.from_numpy(A.n, rp, ci, v)
    with pytest.raises(spai.SpaiError) as ei:
        spai.build_pattern(dA, 0)
    assert ei.value.code == -2
    torch.cuda.synchronize()
