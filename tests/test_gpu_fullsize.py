"""Full-size checks, in the launch configuration the benchmark times.

3D diffusion on 128^3 cells (n = 2,097,152, nnz = 14,581,760), GNN-built G
(Sec. 3.2.2) in float32 storage, eps = 0.3, float32 PCG in float64
refinement to ||b - A x|| / ||b|| <= 1e-8 (Algorithm 1, Sec. 4.2):
* pattern and transpose bit-exact against the oracle on every entry;
* G on sampled rows against the oracle's forward pass on each row's
  (L + 1)-hop neighbourhood (exact by the locality of Eq. 4, pinned on the
  CPU in test_oracle_gnn.py), same tolerance as the small-size GNN tests;
* the solve's x: the oracle's float64 true residual meets the tolerance.

Graph Laplacian with n = 10^6, 8 * 10^6 edges: mixed and float64 solves both
meet the tolerance by the oracle's residual, and their distance is bounded
by what two solutions at that residual may differ by.

A batch of uneven anisotropic systems: every result in the batch is the
same as the system solved alone and meets the tolerance."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import gnn, pattern, pcg
from tests.ball import ball, entries_of_rows, submatrix

pytestmark = pytest.mark.gpu
TOL_G = 2e-5


def upload(spai, A):
    return spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)


@pytest.fixture(scope="module")
def diffusion128():
    A, k = W.diffusion3d(128, 1.5, 8.0, seed=W.BASE_SEED + 2)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, 4, seed=W.BASE_SEED + 100)
    b = W.rhs_uniform(A.n, W.BASE_SEED + 10)
    return A, v, blob, b


def test_diffusion128_pattern_gnn_and_solve(spai_lib, diffusion128):
    spai = spai_lib
    A, v, blob, b = diffusion128
    assert (A.n, A.nnz) == (2_097_152, 14_581_760)
    dA = upload(spai, A)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    out = {key: t.cpu().numpy() for key, t in P.export().items()}
    trp, tci, perm = pattern.transpose_fast(A.n, A.rowptr, A.colidx)
    assert np.array_equal(out["rowptr"], A.rowptr) and np.array_equal(out["colidx"], A.colidx)
    assert np.array_equal(out["t_rowptr"], trp) and np.array_equal(out["t_colidx"], tci)
    assert np.array_equal(out["perm"], perm)

    M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"), torch.tensor(blob, device="cuda"), d_node=4,
                         n_layers=4, g_dtype=spai.F32, eps=0.3)
    g_dev, gt_dev = (t.cpu().numpy() for t in M.export(spai.F64))
    assert np.array_equal(gt_dev[perm], g_dev)           # G^T values are G's, moved by perm
    nrm = gnn.matrix_norm(A.val)
    assert abs(M.matrix_norm() - nrm) <= 1e-12 * nrm
    rs = np.random.default_rng(W.BASE_SEED + 77)
    seeds = np.sort(rs.choice(A.n, size=24, replace=False))
    seeds = np.concatenate([seeds, [0, A.n - 1]])        # two corner cells (boundary rows)
    for grp in np.array_split(seeds, 6):
        nodes = ball(A, grp, 5)
        sub, ent = submatrix(A, nodes)
        g_ref = gnn.gnn_forward(sub.n, sub.rowptr, sub.colidx, sub.val, v[nodes], blob, a_norm=nrm)
        mine = entries_of_rows(sub, np.searchsorted(nodes, grp))
        want, got = g_ref[mine], g_dev[ent[mine]]
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= TOL_G, err

    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, precision=spai.PREC_MIXED, rtol=1e-8,
                       inner_rtol=0.1, max_iter=400000)
    assert r["status"] == 0, r
    xh = x.cpu().numpy()
    rel = pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, xh, b)
    assert rel <= 1e-8, rel
    assert abs(rel - r["true_rel_res"]) <= 1e-3 * rel   # the library's own float64 check agrees


def test_graph_laplacian_1m_mixed_and_f64(spai_lib):
    spai = spai_lib
    A = W.graph_laplacian(1_000_000, 8_000_000)
    assert A.nnz == 17_000_000
    v = W.row_average_feature(A)
    blob = W.gnn_random_weights(1, 4, seed=W.BASE_SEED + 100)
    b = W.rhs_normal(A.n, W.BASE_SEED + 30)
    dA = upload(spai, A)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    feat = torch.tensor(v.reshape(-1, 1).astype(np.float32), device="cuda")
    wts = torch.tensor(blob, device="cuda")
    xs = {}
    for prec, gdt in ((spai.PREC_MIXED, spai.F32), (spai.PREC_F64, spai.F64)):
        M = spai.gnn_precond(dA, P, feat, wts, d_node=1, n_layers=4, g_dtype=gdt, eps=0.3)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, precision=prec, rtol=1e-8, max_iter=100000)
        assert r["status"] == 0, r
        xs[prec] = x.cpu().numpy()
        assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, xs[prec], b) <= 1e-8
    # two solutions with relative residual <= 1e-8 differ by at most
    # 2e-8 * ||A^-1|| ||b|| / ||x||, and ||A^-1|| <= 1 / shift
    diag = A.val[A.colidx == np.repeat(np.arange(A.n), np.diff(A.rowptr))]
    shift = 1e-4 * (diag.mean() / (1 + 1e-4))
    x64 = xs[spai.PREC_F64]
    bound = 2e-8 * np.linalg.norm(b) / shift / np.linalg.norm(x64)
    assert np.linalg.norm(xs[spai.PREC_MIXED] - x64) / np.linalg.norm(x64) <= bound


def test_aniso_batch_alone_equals_batch(spai_lib):
    spai = spai_lib
    mats = [W.aniso2d(N, a, th) for N, a, th in W.aniso2d_batch(12, side_lo=32, side_hi=160)]
    blob = W.gnn_random_weights(1, 4, seed=W.BASE_SEED + 100)
    wts = torch.tensor(blob, device="cuda")
    systems, preconds, bs, alone = [], [], [], []
    for i, A in enumerate(mats):
        dA = upload(spai, A)
        P = spai.build_pattern(dA, spai.PATTERN_FULL)
        feat = torch.tensor(W.row_average_feature(A).reshape(-1, 1).astype(np.float32), device="cuda")
        M = spai.gnn_precond(dA, P, feat, wts, d_node=1, n_layers=4, g_dtype=spai.F32, eps=0.3)
        S = spai.system_create(dA)
        b = torch.tensor(W.rhs_uniform(A.n, W.BASE_SEED + 40 + i), device="cuda")
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = spai.system_solve(S, M, b, x, precision=spai.PREC_MIXED, rtol=1e-8, max_iter=200000)
        assert r["status"] == 0
        alone.append((r, x.clone()))
        systems.append(S), preconds.append(M), bs.append(b)
    xs = [torch.zeros_like(x) for _, x in alone]
    res = spai.pcg_solve_batched(systems, preconds, bs, xs, precision=spai.PREC_MIXED, rtol=1e-8, max_iter=200000)
    for A, (ra, xa), rb, xb, b in zip(mats, alone, res, xs, bs):
        assert rb["status"] == 0 and rb["iters"] == ra["iters"] and rb["outer_iters"] == ra["outer_iters"]
        assert torch.equal(xa, xb)
        assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, xb.cpu().numpy(), b.cpu().numpy()) <= 1e-8


def test_paper_synthetic_ppt_gnn_and_solve(spai_lib):
    # the paper's synthetic family A = P P^T + 1e-4 I (App. C), row-average
    # node feature: pattern exact, G against the oracle, mixed solve to 1e-8
    from oracle import pattern as Pt
    spai = spai_lib
    A = W.ppt_synthetic(3000, seed=W.BASE_SEED + 60)
    dA = upload(spai, A)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    out = {key: t.cpu().numpy() for key, t in P.export().items()}
    trp, tci, perm = Pt.transpose_fast(A.n, A.rowptr, A.colidx)
    assert np.array_equal(out["perm"], perm) and np.array_equal(out["t_colidx"], tci)
    v = W.row_average_feature(A)
    blob = W.gnn_random_weights(1, 4, seed=W.BASE_SEED + 100)
    M = spai.gnn_precond(dA, P, torch.tensor(v.reshape(-1, 1).astype(np.float32), device="cuda"),
                         torch.tensor(blob, device="cuda"), d_node=1, n_layers=4, g_dtype=spai.F32, eps=0.3)
    g, _ = M.export(spai.F64)
    ref = gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, blob)
    g = g.cpu().numpy()
    assert np.abs(g - ref).max() <= TOL_G * np.abs(ref).max()
    b = W.rhs_uniform(A.n, W.BASE_SEED + 61)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, precision=spai.PREC_MIXED, rtol=1e-8,
                       max_iter=200000)
    assert r["status"] == 0
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.cpu().numpy(), b) <= 1e-8
