"""The GNN reverse pass of the CUDA library, run by a host executor of the
same driver and element functions (tests/gnn_grad_host.cpp, built here with
g++), against the oracle's reverse pass (itself pinned by central
differences in test_oracle_train.py)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as W
from oracle import gnn, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_LIB = None


def host_lib():
    global _LIB
    if _LIB is None:
        out = os.path.join(tempfile.mkdtemp(prefix="gnn_grad_host_"), "libgnn_grad_host.so")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                               "-I", os.path.join(ROOT, "paper_2510_27517_gb300", "csrc"),
                               os.path.join(ROOT, "tests", "gnn_grad_host.cpp"), "-o", out])
        _LIB = ctypes.CDLL(out)
        _LIB.gnn_grad_host.restype = ctypes.c_int
    return _LIB


def host_grad(A, v, blob, n_layers, raw, dg, b=1):
    P = ctypes.c_void_p
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
    av = np.ascontiguousarray(A.val, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    w = np.ascontiguousarray(blob, dtype=np.float64)
    dg = np.ascontiguousarray(dg, dtype=np.float64)
    out = np.zeros_like(w)
    rc = host_lib().gnn_grad_host(ctypes.c_int64(A.n), P(rp.ctypes.data), P(ci.ctypes.data), P(av.ctypes.data),
                                  P(vv.ctypes.data), ctypes.c_int(vv.shape[1]), P(w.ctypes.data),
                                  ctypes.c_int(n_layers), ctypes.c_int(int(raw)), ctypes.c_int(b),
                                  P(dg.ctypes.data), P(out.ctypes.data))
    assert rc == 0, rc
    return out


@pytest.mark.parametrize("raw", [False, True])
@pytest.mark.parametrize("n_layers", [0, 1, 3])
def test_host_executor_matches_oracle_reverse_pass(raw, n_layers):
    A = W.random_spd_sparse(40, 0.12, 23)
    v = np.random.default_rng(1).uniform(-1, 1, size=(A.n, 3))
    blob = W.gnn_random_weights(3, n_layers, seed=31, msg_raw_edge=raw).astype(np.float64) * 1.5
    dg = np.random.default_rng(2).standard_normal(A.nnz)
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v, blob, n_layers, raw)
    want = train.gnn_backward(tape, dg)
    got = host_grad(A, v, blob, n_layers, raw, dg)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_host_executor_sai_chain_on_a_stencil():
    # dL/dG of the SAI loss (oracle) pushed through the host executor equals
    # the oracle's full gradient in the weights
    A, k = W.diffusion3d(4)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, 2, seed=7).astype(np.float64)
    w = np.random.default_rng(9).standard_normal((A.n, 3))
    g, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v, blob, 2)
    _, dg = train.sai_loss_grad_g(A.n, A.rowptr, A.colidx, A.val, A.rowptr, A.colidx, g, 0.1, w)
    _, want = train.loss_and_grad(A.n, A.rowptr, A.colidx, A.val, v, blob, 0.1, w, n_layers=2)
    got = host_grad(A, v, blob, 2, False, dg)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_host_executor_paper_configuration():
    # the paper's configuration: 4 layers, d_node 4, latent messages, on a 3D
    # diffusion stencil with its position + log-coefficient node features
    A, k = W.diffusion3d(6)
    v = W.diffusion3d_node_features(k)
    blob = W.gnn_random_weights(4, 4).astype(np.float64)
    dg = np.random.default_rng(4).standard_normal(A.nnz)
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, v, blob, 4)
    want = train.gnn_backward(tape, dg)
    got = host_grad(A, v, blob, 4, False, dg)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # every MLP receives a gradient (units whose ReLU is off everywhere get none)
    o = 0
    for fi, fo in gnn.layer_shapes(4, 4):
        size = gnn.HIDDEN * fi + gnn.HIDDEN + fo * gnn.HIDDEN + fo
        assert np.abs(got[o:o + size]).max() > 0
        o += size


def test_host_executor_rejects_unsymmetric_pattern():
    A = W.random_spd_sparse(10, 0.3, 2)
    keep = np.ones(A.nnz, dtype=bool)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = np.nonzero(A.colidx != rows)[0]
    keep[off[0]] = False  # drop one off-diagonal entry: (i, j) stays, (j, i) goes
    B = W.coo_to_csr(A.n, rows[keep], A.colidx[keep], A.val[keep])
    rp = np.ascontiguousarray(B.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(B.colidx, dtype=np.int32)
    av = np.ascontiguousarray(B.val)
    v = np.zeros((B.n, 1))
    w = W.gnn_random_weights(1, 1).astype(np.float64)
    dg = np.zeros(B.nnz)
    out = np.zeros_like(w)
    P = ctypes.c_void_p
    rc = host_lib().gnn_grad_host(ctypes.c_int64(B.n), P(rp.ctypes.data), P(ci.ctypes.data), P(av.ctypes.data),
                                  P(v.ctypes.data), ctypes.c_int(1), P(w.ctypes.data), ctypes.c_int(1),
                                  ctypes.c_int(0), ctypes.c_int(1), P(dg.ctypes.data), P(out.ctypes.data))
    assert rc == -1


@pytest.mark.parametrize("raw", [False, True])
def test_host_executor_block_gnn(raw):
    # 3 x 3 blocks: the GNN on the node graph, 9-wide edge features and
    # decoder output, the gradient gathered from the scalar CSR order
    A, feat = W.elastic3d(3)
    blob = W.gnn_random_weights(4, 2, seed=41, msg_raw_edge=raw, b=3).astype(np.float64) * 1.5
    dg = np.random.default_rng(6).standard_normal(A.nnz)
    _, tape = train.gnn_forward_tape(A.n, A.rowptr, A.colidx, A.val, feat, blob, 2, raw, b=3)
    want = train.gnn_backward(tape, dg)
    got = host_grad(A, feat, blob, 2, raw, dg, b=3)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
