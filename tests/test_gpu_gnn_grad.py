"""The GNN reverse pass on the GPU (spai_gnn_grad: Sec. 3.3 trains the GNN of
Sec. 3.2.2, Eqs. 3-5, on the SAI loss) against the oracle's reverse pass,
which test_oracle_train.py pins by central differences.

Both sides run in float64 from the same float32 weights and features; they
differ only in summation order (the GPU sums weight gradients in fixed
chunks), so the bar is 1e-10 of the largest gradient entry.  Also: inputs a
3 x 3 block GNN must reject."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import train

pytestmark = pytest.mark.gpu
TOL = 1e-10


def gpu_grad(spai, A, v, blob, dg, d_node, L, raw=False, b=1):
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    out = spai.gnn_grad(dA, P, torch.tensor(np.asarray(v, np.float32), device="cuda").contiguous(),
                        torch.tensor(np.asarray(blob, np.float32), device="cuda"),
                        torch.tensor(dg, dtype=torch.float64, device="cuda"), d_node=d_node, n_layers=L,
                        msg_edge=spai.MSG_RAW if raw else spai.MSG_LATENT, block=b)
    return out.cpu().numpy()


def oracle_grad(A, v, blob, dg, L, raw=False, b=1):
    # the oracle reads the float32 inputs the GPU reads, widened to float64
    v64 = np.asarray(v, np.float32).astype(np.float64)
    w64 = np.asarray(blob, np.float32).astype(np.float64)
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v64, w64, L, raw, b=b)
    return train.gnn_backward(tape, dg)


def rel_err(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("raw", [False, True])
@pytest.mark.parametrize("L", [0, 1, 4])
def test_scalar_gnn_grad_matches_oracle(spai_lib, raw, L):
    A, k = W.diffusion3d(4)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, L, seed=17, msg_raw_edge=raw) * 1.5
    dg = np.random.default_rng(5).standard_normal(A.nnz)
    got = gpu_grad(spai_lib, A, v, blob, dg, 4, L, raw)
    want = oracle_grad(A, v, blob, dg, L, raw)
    assert got.shape == want.shape
    assert rel_err(got, want) <= TOL, rel_err(got, want)


def test_scalar_gnn_grad_16cube_paper_configuration(spai_lib):
    # 4 layers, latent messages, position + log-coefficient features, 16^3
    A, k = W.diffusion3d(16)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, 4, seed=3)
    dg = np.random.default_rng(8).standard_normal(A.nnz)
    got = gpu_grad(spai_lib, A, v, blob, dg, 4, 4)
    want = oracle_grad(A, v, blob, dg, 4)
    assert rel_err(got, want) <= TOL, rel_err(got, want)


def test_graph_laplacian_gnn_grad(spai_lib):
    # irregular rows (average 17 entries, long tails) and a 1-wide feature
    A = W.graph_laplacian(600, 4800, seed=4)
    v = W.row_average_feature(A)
    blob = W.gnn_random_weights(1, 2, seed=9)
    dg = np.random.default_rng(2).standard_normal(A.nnz)
    got = gpu_grad(spai_lib, A, v, blob, dg, 1, 2)
    want = oracle_grad(A, v, blob, dg, 2)
    assert rel_err(got, want) <= TOL, rel_err(got, want)


@pytest.mark.parametrize("raw", [False, True])
def test_block_gnn_grad_matches_oracle(spai_lib, raw):
    A, feat = W.elastic3d(3)
    blob = W.gnn_random_weights(feat.shape[1], 2, seed=41, msg_raw_edge=raw, b=3) * 1.5
    dg = np.random.default_rng(6).standard_normal(A.nnz)
    got = gpu_grad(spai_lib, A, feat, blob, dg, feat.shape[1], 2, raw, b=3)
    want = oracle_grad(A, feat, blob, dg, 2, raw, b=3)
    assert rel_err(got, want) <= TOL, rel_err(got, want)


def test_sai_chain_on_the_gpu(spai_lib):
    # dL/dG of the SAI loss (spai_sai_loss_grad) pushed through the reverse
    # pass equals the oracle's gradient of the loss in the weights
    spai = spai_lib
    A, k = W.diffusion3d(5)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, 2, seed=7)
    w = np.random.default_rng(9).standard_normal((A.n, 3))
    eps = 0.1
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    vt = torch.tensor(v.astype(np.float32), device="cuda")
    bt = torch.tensor(blob.astype(np.float32), device="cuda")
    M = spai.gnn_precond(dA, P, vt, bt, d_node=4, n_layers=2, g_dtype=spai.F64, eps=eps)
    _, dg = spai.sai_loss_grad(dA, M, torch.tensor(w, device="cuda"))
    got = spai.gnn_grad(dA, P, vt, bt, dg, d_node=4, n_layers=2).cpu().numpy()
    _, want = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v.astype(np.float32).astype(np.float64),
                                  blob.astype(np.float32).astype(np.float64), eps, w, n_layers=2)
    # G on the GPU is the float32 forward pass (R12), the oracle's is float64:
    # the gradients agree to the forward pass's float32 tolerance
    assert rel_err(got, want) <= 1e-4, rel_err(got, want)


def _drop_pair(A, i, j):
    """A without the entries (i, j) and (j, i) (pattern stays symmetric)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    keep = ~(((rows == i) & (A.colidx == j)) | ((rows == j) & (A.colidx == i)))
    assert keep.sum() == A.nnz - 2
    return W.coo_to_csr(A.n, rows[keep], A.colidx[keep], A.val[keep])


def _circulant9():
    """9 x 9 periodic tridiagonal SPD matrix: every row has 3 entries and the
    block-row offsets are multiples of 9, but the column runs are not aligned
    to 3 x 3 blocks."""
    n = 9
    rows = np.repeat(np.arange(n), 3)
    cols = np.stack([(np.arange(n) - 1) % n, np.arange(n), (np.arange(n) + 1) % n], 1).ravel()
    vals = np.where(rows == cols, 3.0, -1.0)
    return W.coo_to_csr(n, rows, cols, vals)


@pytest.mark.parametrize("case", ["row_length", "unequal_rows", "misaligned_columns"])
def test_block_gnn_grad_rejects_non_block_inputs(spai_lib, case):
    spai = spai_lib
    A, feat = W.elastic3d(2)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    if case == "row_length":
        # the first scalar row of block row 0 loses an off-block entry: its length is not a multiple of 3
        j = int(A.colidx[(rows == 0) & (A.colidx >= 3)][0])
        B = _drop_pair(A, 0, j)
    elif case == "unequal_rows":
        # the second scalar row of block row 0 loses one: the rows of the block row differ in length
        j = int(A.colidx[(rows == 1) & (A.colidx >= 3)][0])
        B = _drop_pair(A, 1, j)
    else:
        B = _circulant9()
        feat = np.zeros((3, feat.shape[1]))
    blob = W.gnn_random_weights(feat.shape[1], 1, seed=1, b=3)
    dB = spai.CSRMatrix.from_numpy(B.n, B.rowptr, B.colidx, B.val)
    P = spai.build_pattern(dB, spai.PATTERN_FULL)
    with pytest.raises(spai.SpaiError) as ei:
        spai.gnn_grad(dB, P, torch.tensor(feat.astype(np.float32), device="cuda"),
                      torch.tensor(blob.astype(np.float32), device="cuda"),
                      torch.zeros(B.nnz, dtype=torch.float64, device="cuda"), d_node=feat.shape[1], n_layers=1,
                      block=3)
    assert ei.value.code == spai.spai.ERR_SHAPE
