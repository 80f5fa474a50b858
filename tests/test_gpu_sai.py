"""SAI loss (Sec. 3.3, Eqs. 7-8) on the GPU against the float64 oracle, for
GNN-built and classical factors in every storage type."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fsai, sai, train

pytestmark = pytest.mark.gpu


def probes(n, k, seed):
    return np.random.default_rng(seed).standard_normal((n, k))


@pytest.mark.parametrize("gdt", [0, 1, 2, 3])
@pytest.mark.parametrize("k", [1, 7, 32])
def test_gnn_factor_matches_oracle(spai_lib, gdt, k):
    spai = spai_lib
    A, kf = W.diffusion3d(10)
    v = W.diffusion3d_node_features(kf)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"), torch.tensor(W.gnn_random_weights(4, 4), device="cuda"),
                         d_node=4, g_dtype=gdt, eps=0.3)
    g, _ = M.export(spai.F64)
    w = probes(A.n, k, 5 + k)
    got = spai.sai_loss(dA, M, torch.tensor(w, device="cuda")).cpu().numpy()
    want = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g.cpu().numpy(), 0.3, w)
    assert np.allclose(got, want, rtol=1e-11, atol=0)


def test_fsai_factor_and_unit_probes(spai_lib):
    # classical factor on the upper pattern; unit probes sum to ||A M^-1/||A|| - I||_F^2
    spai = spai_lib
    A = W.poisson2d(5)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, spai.PATTERN_UPPER)
    M = spai.precond_from_values(pat, torch.tensor(gv, device="cuda"), spai.F64, eps=0.01)
    w = np.eye(A.n)
    got = np.concatenate([spai.sai_loss(dA, M, torch.tensor(w[:, j:j + 25].copy(), device="cuda")).cpu().numpy()
                          for j in range(0, A.n, 25)])
    want = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, urp, uci, gv, 0.01, w)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("gdt", [0, 1, 2])
def test_loss_gradient_matches_oracle(spai_lib, gdt):
    # gradient of the mean loss over the probes with respect to G's stored
    # values (the training step's first link, Sec. 3.3), GNN factor
    spai = spai_lib
    A, kf = W.diffusion3d(9)
    v = W.diffusion3d_node_features(kf)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"), torch.tensor(W.gnn_random_weights(4, 4), device="cuda"),
                         d_node=4, g_dtype=gdt, eps=0.3)
    g = M.export(spai.F64)[0].cpu().numpy()
    w = probes(A.n, 5, 17)
    loss, grad = spai.sai_loss_grad(dA, M, torch.tensor(w, device="cuda"))
    want_loss, want_grad = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, 0.3, w)
    assert loss.cpu().numpy().mean() == pytest.approx(want_loss, rel=1e-11)
    grad = grad.cpu().numpy()
    assert np.abs(grad - want_grad).max() <= 1e-11 * np.abs(want_grad).max()


def test_fsai_loss_gradient_matches_oracle(spai_lib):
    # a factor on the upper pattern: G's CSR differs from A's
    spai = spai_lib
    A = W.aniso2d(13, 30.0, 0.5)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, spai.PATTERN_UPPER)
    M = spai.precond_from_values(pat, torch.tensor(gv, device="cuda"), spai.F64, eps=0.02)
    w = probes(A.n, 32, 3)
    loss, grad = spai.sai_loss_grad(dA, M, torch.tensor(w, device="cuda"))
    want_loss, want_grad = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, urp, uci, gv, 0.02, w)
    assert loss.cpu().numpy().mean() == pytest.approx(want_loss, rel=1e-11)
    assert np.abs(grad.cpu().numpy() - want_grad).max() <= 1e-11 * np.abs(want_grad).max()


def test_sai_loss_errors(spai_lib):
    spai = spai_lib
    A = W.poisson2d(4)
    dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.precond_from_values(P, torch.ones(A.nnz, dtype=torch.float64, device="cuda"), spai.F64, eps=0.0)
    with pytest.raises(spai.SpaiError):
        spai.sai_loss(dA, M, torch.zeros(A.n, 33, dtype=torch.float64, device="cuda"))
    B = W.poisson2d(5)
    dB = spai.CSRMatrix.from_numpy(B.n, B.rowptr, B.colidx, B.val)
    with pytest.raises(spai.SpaiError):
        spai.sai_loss(dB, M, torch.zeros(B.n, 2, dtype=torch.float64, device="cuda"))
