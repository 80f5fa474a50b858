"""Pins of the training-gradient oracle (Sec. 3.3: the GNN is trained on the
SAI loss of Eqs. 7-8 with probe vectors w ~ N(0, I)).

The loss is a quartic polynomial in G, so central differences pin dL/dG to
near rounding; the reverse pass through the GNN is pinned by central
differences of the forward pass, by a closed form for a constant factor and
by the scale invariance the paper states for ||A||-normalised inputs."""
import numpy as np
import pytest

import workloads as W
from oracle import gnn, sai, spectrum, train


def _system(n=14, seed=3):
    A = W.random_spd_sparse(n, 0.3, seed)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(A.nnz) * 0.3 + np.where(
        A.colidx == np.repeat(np.arange(A.n), np.diff(A.rowptr)), 1.0, 0.0)
    w = rng.standard_normal((A.n, 3))
    return A, g, w


def test_loss_matches_forward_oracle():
    A, g, w = _system()
    loss, _ = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, 0.05, w)
    per = sai.sai_loss(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, 0.05, w)
    assert loss == pytest.approx(per.mean(), rel=1e-14)


@pytest.mark.parametrize("eps", [0.0, 0.2])
def test_grad_g_matches_central_differences(eps):
    # every stored entry; G is not symmetric, so a transposed index fails
    A, g, w = _system()
    f = lambda gv: train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, gv, eps, w)[0]  # noqa
    _, grad = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, eps, w)
    h = 1e-5
    fd = np.empty_like(g)
    for e in range(g.size):
        gp, gm = g.copy(), g.copy()
        gp[e] += h
        gm[e] -= h
        fd[e] = (f(gp) - f(gm)) / (2 * h)
    assert np.abs(fd - grad).max() <= 1e-7 * np.abs(grad).max()


def test_grad_g_dense_closed_form():
    # dL/dG = (2/k) sum_w [a (G^T w)^T + w (G^T a)^T] on the pattern, with
    # a = A^T E w / ||A||: written with dense matrices, restricted to the pattern
    A, g, w = _system(10, 7)
    eps = 0.1
    a_d = spectrum.dense_from_csr(A.n, A.rowptr, A.colidx, A.val)
    g_d = spectrum.dense_from_csr(A.n, A.rowptr, A.colidx, g)
    nrm = gnn.matrix_norm(A.val)
    E = a_d @ (g_d @ g_d.T + eps * np.eye(A.n)) / nrm - np.eye(A.n)
    full = np.zeros_like(g_d)
    for p in range(w.shape[1]):
        wp = w[:, p]
        a = a_d.T @ (E @ wp) / nrm
        full += 2.0 * (np.outer(a, g_d.T @ wp) + np.outer(wp, g_d.T @ a))
    full /= w.shape[1]
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    _, grad = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, eps, w)
    assert np.allclose(grad, full[rows, A.colidx], rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_grad_g_scaled_identity():
    # A = c I, G = alpha I, eps = 0: E = (alpha^2 - 1) I, so
    # L = (alpha^2 - 1)^2 |w|^2 and dL/dG_ii = 4 alpha (alpha^2 - 1) w_i^2
    n, c, alpha = 6, 3.0, 0.8
    rp, ci = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32)
    w = np.random.default_rng(1).standard_normal((n, 1))
    loss, grad = train.sai_loss_grad_g(n, rp, ci, np.full(n, c), rp, ci, np.full(n, alpha), 0.0, w)
    assert loss == pytest.approx((alpha ** 2 - 1) ** 2 * float(w[:, 0] @ w[:, 0]), rel=1e-14)
    assert np.allclose(grad, 4 * alpha * (alpha ** 2 - 1) * w[:, 0] ** 2, rtol=1e-14)


def _graph(n=7, seed=11):
    A = W.random_spd_sparse(n, 0.5, seed)
    v = np.random.default_rng(seed).uniform(-1, 1, size=(A.n, 2))
    blob = W.gnn_random_weights(2, 2, seed=seed).astype(np.float64) * 1.5
    return A, v, blob


@pytest.mark.parametrize("raw", [False, True])
def test_tape_forward_is_the_forward_oracle(raw):
    A, v, _ = _graph()
    blob = W.gnn_random_weights(2, 2, seed=5, msg_raw_edge=raw).astype(np.float64)
    g_ref = gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, blob, n_layers=2, msg_raw_edge=raw)
    g, _ = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v, blob, n_layers=2, msg_raw_edge=raw)
    assert np.array_equal(g, g_ref)


@pytest.mark.parametrize("raw", [False, True])
def test_gnn_backward_matches_central_differences(raw):
    # objective s . G for a fixed random s; every weight and bias of the blob
    A, v, _ = _graph()
    blob = W.gnn_random_weights(2, 2, seed=9, msg_raw_edge=raw).astype(np.float64) * 1.5
    s = np.random.default_rng(2).standard_normal(A.nnz)
    f = lambda b: float(s @ gnn.gnn_forward(A.n, A.rowptr, A.colidx, A.val, v, b, 2, raw))  # noqa: E731
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v, blob, 2, raw)
    grad = train.gnn_backward(tape, s)
    assert grad.shape == blob.shape
    h = 1e-6
    fd = np.empty_like(blob)
    for k in range(blob.size):
        bp, bm = blob.copy(), blob.copy()
        bp[k] += h
        bm[k] -= h
        fd[k] = (f(bp) - f(bm)) / (2 * h)
    assert np.abs(fd - grad).max() <= 1e-6 * np.abs(grad).max()
    # the check is not vacuous: every MLP of the blob gets a gradient
    o = 0
    for fi, fo in gnn.layer_shapes(2, 2, raw):
        size = gnn.HIDDEN * fi + gnn.HIDDEN + fo * gnn.HIDDEN + fo
        assert np.abs(grad[o:o + size]).max() > 0
        o += size


def test_full_chain_matches_central_differences():
    A, v, blob = _graph(8, 13)
    w = np.random.default_rng(4).standard_normal((A.n, 2))
    eps = 0.05
    loss, grad = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, blob, eps, w, n_layers=2)
    f = lambda b: train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, b, eps, w, n_layers=2)[0]  # noqa: E731
    assert f(blob) == loss
    pick = np.random.default_rng(6).choice(blob.size, 60, replace=False)
    h = 1e-6
    for k in pick:
        bp, bm = blob.copy(), blob.copy()
        bp[k] += h
        bm[k] -= h
        fd = (f(bp) - f(bm)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * np.abs(grad).max(), k


def test_constant_factor_gradient():
    # all weights zero but the decoder's output bias c: G = c everywhere, the
    # only nonzero gradient is d/dc = sum over the stored entries of dL/dG_ij
    A, v, _ = _graph()
    blob = np.zeros(W.gnn_param_count(2, 2))
    blob[-1] = 0.4
    w = np.random.default_rng(8).standard_normal((A.n, 2))
    loss, grad = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, blob, 0.1, w, n_layers=2)
    _, dg = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, np.full(A.nnz, 0.4), 0.1, w)
    assert grad[-1] == pytest.approx(dg.sum(), rel=1e-13)
    assert np.count_nonzero(grad[:-1]) == 0


def test_scale_invariance_of_loss_and_gradient():
    # the GNN sees A / ||A|| and the loss uses A / ||A||: scaling A changes neither
    A, v, blob = _graph()
    w = np.random.default_rng(3).standard_normal((A.n, 2))
    l1, g1 = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, blob, 0.05, w, n_layers=2)
    l2, g2 = train.loss_and_grad(A.n, A.rowptr, A.colidx, 37.5 * A.val, v, blob, 0.05, w, n_layers=2)
    assert l2 == pytest.approx(l1, rel=1e-12)
    assert np.allclose(g2, g1, rtol=1e-10, atol=1e-12 * np.abs(g1).max())


def test_gradient_steps_lower_the_loss():
    # gradient descent with step halving on one system with fixed probes: the
    # negative gradient is a descent direction at every step (a wrong sign or
    # a dropped term shows up as a step that cannot lower the loss)
    A, v, blob = _graph(10, 17)
    w = np.random.default_rng(5).standard_normal((A.n, 4))
    f = lambda b: train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, b, 0.05, w, n_layers=2)  # noqa: E731
    loss, grad = f(blob)
    first = loss
    for _ in range(6):
        t = 0.05 / np.abs(grad).max()
        for _ in range(40):
            cand, cgrad = f(blob - t * grad)
            if cand < loss:
                break
            t *= 0.5
        assert cand < loss
        blob, loss, grad = blob - t * grad, cand, cgrad
    assert loss < 0.5 * first


def _blocks():
    A, feat = W.elastic3d(2)
    blob = W.gnn_random_weights(4, 2, seed=21, b=3).astype(np.float64) * 1.5
    return A, feat, blob


def test_block_tape_forward_is_the_block_forward_oracle():
    A, feat, blob = _blocks()
    ref = gnn.gnn_forward_blocks(A.n, A.rowptr, A.colidx, A.val, feat, blob, 3, n_layers=2)
    g, _ = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, feat, blob, n_layers=2, b=3)
    assert np.array_equal(g, ref)


def test_block_gnn_backward_matches_central_differences():
    # 3 x 3 blocks: the decoder writes 9 values per block edge, scattered to
    # the scalar CSR; the reverse pass gathers them back
    A, feat, blob = _blocks()
    s = np.random.default_rng(12).standard_normal(A.nnz)
    f = lambda b: float(s @ gnn.gnn_forward_blocks(A.n, A.rowptr, A.colidx, A.val, feat, b, 3, n_layers=2))  # noqa
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, feat, blob, n_layers=2, b=3)
    grad = train.gnn_backward(tape, s)
    assert grad.shape == blob.shape
    # every decoder output weight and bias, and a sample of the rest
    dec = gnn.HIDDEN * gnn.HIDDEN + gnn.HIDDEN + 9 * gnn.HIDDEN + 9
    pick = np.concatenate([np.arange(blob.size - dec, blob.size),
                           np.random.default_rng(13).choice(blob.size - dec, 120, replace=False)])
    h = 1e-6
    for k in pick:
        bp, bm = blob.copy(), blob.copy()
        bp[k] += h
        bm[k] -= h
        fd = (f(bp) - f(bm)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * np.abs(grad).max(), k


def test_block_full_chain_matches_central_differences():
    A, feat, blob = _blocks()
    w = np.random.default_rng(14).standard_normal((A.n, 2))
    loss, grad = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, feat, blob, 0.05, w, n_layers=2, b=3)
    f = lambda b: train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, feat, b, 0.05, w, n_layers=2, b=3)[0]  # noqa
    pick = np.random.default_rng(15).choice(blob.size, 40, replace=False)
    h = 1e-6
    for k in pick:
        bp, bm = blob.copy(), blob.copy()
        bp[k] += h
        bm[k] -= h
        fd = (f(bp) - f(bm)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * np.abs(grad).max(), k
