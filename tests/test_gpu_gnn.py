"""GNN forward on the GPU (Sec. 3.2.2, Eqs. 3-5) against the float64 oracle.

The GPU computes in float32 with the first-layer split; the tolerance
(relative to max |G|) is 2e-5 per the float32 rounding of ~10 chained
24-term dot products (about 10 * 24 * 2^-24 relative growth)."""
import json
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import gnn
from tests.weights_util import blob_from_entries

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 2e-5


def run_gpu(spai, A, v, blob, d_node, L=4, raw=False, g_dtype=1, eps=1e-4):
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(np.asarray(v, np.float32), device="cuda").contiguous(),
                         torch.tensor(blob, device="cuda"), d_node=d_node, n_layers=L,
                         msg_edge=spai.MSG_RAW if raw else spai.MSG_LATENT, g_dtype=g_dtype, eps=eps)
    g, gt = M.export(spai.F64)
    return M, g.cpu().numpy(), gt.cpu().numpy()


def test_hand_computed_golden(spai_lib):
    fx = json.load(open(os.path.join(GOLDEN, "gnn_path3_one_layer.json")))
    blob, _ = blob_from_entries(fx["d_node"], fx["n_layers"], fx["weights_nonzero"])
    A = W.CSR(fx["n"], np.array(fx["rowptr"], np.int32), np.array(fx["colidx"], np.int32), np.array(fx["aval"]))
    _, g, gt = run_gpu(spai_lib, A, np.array(fx["node_feat"]), blob, 1, L=1)
    assert np.allclose(g, fx["expected_g"], rtol=1e-6)


@pytest.mark.parametrize("L", [0, 1, 4])
@pytest.mark.parametrize("raw", [False, True])
def test_diffusion_matches_oracle(spai_lib, L, raw):
    A, k = W.diffusion3d(10)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, L, seed=7, msg_raw_edge=raw)
    ref = gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, blob, n_layers=L, msg_raw_edge=raw)
    M, g, gt = run_gpu(spai_lib, A, v, blob, 4, L=L, raw=raw)
    err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    assert err <= TOL, err
    # G^T values are G's, permuted through the mirror entries
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    D = np.zeros((A.n, A.n)); D[rows, A.colidx] = g
    assert np.array_equal(gt, D.T[rows, A.colidx])
    assert M.matrix_norm() == pytest.approx(gnn.matrix_norm(A.val), rel=1e-14)


def test_graph_laplacian_and_long_rows(spai_lib):
    A = W.graph_laplacian(2000, 16000, seed=9)
    # add a hub node connected to 400 others to exercise rows longer than a group
    v = W.row_average_feature(A)
    blob = W.gnn_random_weights(1, 4, seed=3)
    ref = gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, blob)
    _, g, _ = run_gpu(spai_lib, A, v, blob, 1)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) <= TOL

    n = 700
    rows = np.concatenate([np.zeros(n - 1, int), np.arange(1, n), np.arange(n)])
    cols = np.concatenate([np.arange(1, n), np.zeros(n - 1, int), np.arange(n)])
    vals = np.concatenate([-np.ones(2 * (n - 1)) * 0.3, np.full(n, 2.0)])
    vals[-n] = 0.3 * n + 1.0
    H = W.coo_to_csr(n, rows, cols, vals)
    vh = W.row_average_feature(H)
    ref = gnn.gnn_forward(H.n, H.rowptr, H.colidx, H.val, vh, blob)
    _, g, _ = run_gpu(spai_lib, H, vh, blob, 1)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) <= TOL


def test_low_precision_storage(spai_lib):
    A, k = W.diffusion3d(6)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4)
    ref = gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, blob)
    # storage rounding (half an ulp of the format) on top of the float32 compute error
    for gdt, unit in ((0, 0.0), (2, 2.0 ** -8), (3, 2.0 ** -11)):
        _, g, _ = run_gpu(spai_lib, A, v, blob, 4, g_dtype=gdt)
        bound = unit * np.abs(ref) * 1.01 + TOL * np.abs(ref).max()
        assert np.all(np.abs(g - ref) <= bound)


def test_shape_errors(spai_lib):
    spai = spai_lib
    A, k = W.diffusion3d(4)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4)
    with pytest.raises(spai.SpaiError) as ei:
        run_gpu(spai, A, v, blob[:-1], 4)
    assert ei.value.code == -3
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_UPPER)
    with pytest.raises(spai.SpaiError):
        spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"), torch.tensor(blob, device="cuda"), d_node=4)


def test_gnn_then_mixed_solve(spai_lib):
    spai = spai_lib
    A, k = W.diffusion3d(12)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4)
    M, g, _ = run_gpu(spai, A, v, blob, 4, eps=1e-2)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    b = W.rhs_uniform(A.n, 3)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, precision=spai.PREC_MIXED)
    from oracle import pcg
    assert res["status"] == 0
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.cpu().numpy(), b) <= 1e-8


@pytest.mark.parametrize("raw", [False, True])
def test_block_gnn_matches_oracle_and_solves(spai_lib, raw):
    # 3 x 3 blocks (Sec. 3.2.2 with b = 3): node graph, 9-wide edge features
    # and decoder output, G written block by block into A's scalar pattern
    from oracle import pcg
    spai = spai_lib
    A, feat = W.elastic3d(5)
    L = 2 if raw else 4
    blob = W.gnn_random_weights(4, L, msg_raw_edge=raw, b=3)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(feat, device="cuda"), torch.tensor(blob, device="cuda"), d_node=4,
                         n_layers=L, msg_edge=spai.MSG_RAW if raw else spai.MSG_LATENT, g_dtype=spai.F32, eps=0.3,
                         block=3)
    g, gt = (t.cpu().numpy() for t in M.export(spai.F64))
    ref = gnn.gnn_forward_blocks(A.n, A.rowptr, A.colidx, A.val, feat, blob, 3, n_layers=L, msg_raw_edge=raw)
    assert np.abs(g - ref).max() <= TOL * np.abs(ref).max()
    perm = P.export()["perm"].cpu().numpy()
    assert np.array_equal(gt[perm], g)
    b = W.rhs_uniform(A.n, 17)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, precision=spai.PREC_MIXED, rtol=1e-8,
                       max_iter=100000)
    assert r["status"] == 0
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.cpu().numpy(), b) <= 1e-8


def test_block_gnn_rejects_non_block_matrix(spai_lib):
    spai = spai_lib
    A = W.poisson2d(6)                    # 36 rows, but not dense 3 x 3 blocks
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    blob = W.gnn_random_weights(1, 1, b=3)
    with pytest.raises(spai.SpaiError) as ei:
        spai.gnn_precond(dA, P, torch.zeros(12, 1, device="cuda"), torch.tensor(blob, device="cuda"), d_node=1,
                         n_layers=1, g_dtype=spai.F32, eps=0.3, block=3)
    assert ei.value.code == spai.spai.ERR_BAD_CSR
