"""Gradients of the SAI loss for training the GNN (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.3 trains the GNN of Sec. 3.2.2 by minimising the SAI loss, estimated
with standard-normal probe vectors w (Hutchinson's estimator, Eq. 7):

    L(w) = || E w ||^2,   E = A M^-1 / ||A|| - I,   M^-1 = G G^T + eps I (Eq. 1),

averaged over the probes of a batch (the expectation of Eq. 7).  Two steps:

* the gradient with respect to the stored values of G.  With u = E w,
  a = A^T u / ||A||, y = G^T w and c = G^T a, the differential of L(w) is
  2 a^T dG y + 2 w^T dG c, so

      dL/dG_ij = 2 (a_i y_j + w_i c_j)     for every stored (i, j) of G;

* reverse-mode differentiation of the forward pass (Eqs. 3-5) from dL/dG to
  every weight of the blob, layer by layer in the opposite order.  ||A|| and
  the edge features do not depend on the weights.

The forward pass here repeats ``gnn._forward`` operation for operation while
keeping what the reverse pass needs (a test checks that both give the same
G bit for bit); ReLU'(0) is taken as 0.
"""
from __future__ import annotations

import numpy as np

from . import gnn, pcg


# ---- the loss and its gradient with respect to G ----
def sai_loss_grad_g(n, rowptr, colidx, val, g_rowptr, g_colidx, g_val, eps, w):
    """Mean SAI loss over the probes (columns of w, shape (n, k)) and its
    gradient with respect to g_val (G in CSR: row i, column j, value G_ij)."""
    w = np.asarray(w, dtype=np.float64).reshape(n, -1)
    k = w.shape[1]
    nrm = gnn.matrix_norm(val)
    g_rows = np.repeat(np.arange(n), np.diff(np.asarray(g_rowptr, dtype=np.int64)))
    g_cols = np.asarray(g_colidx, dtype=np.int64)
    apply = pcg.spai_apply(n, g_rowptr, g_colidx, g_val, eps)
    loss = 0.0
    grad = np.zeros(len(g_cols))
    for p in range(k):
        wp = w[:, p]
        u = pcg.spmv(n, rowptr, colidx, val, apply(wp)) / nrm - wp          # E w
        a = pcg.spmv_transpose(n, rowptr, colidx, val, u) / nrm             # A^T u / ||A||
        y = pcg.spmv_transpose(n, g_rowptr, g_colidx, g_val, wp)            # G^T w
        c = pcg.spmv_transpose(n, g_rowptr, g_colidx, g_val, a)             # G^T a
        loss += float(u @ u)
        grad += 2.0 * (a[g_rows] * y[g_cols] + wp[g_rows] * c[g_cols])
    return loss / k, grad / k


# ---- one-hidden-layer MLP with its reverse pass ----
def _mlp_fwd(p, z):
    w1, b1, w2, b2 = p
    pre = z @ w1.T + b1
    hid = np.maximum(pre, 0.0)
    return hid @ w2.T + b2, (z, pre, hid)


def _mlp_bwd(p, cache, dy, grads):
    """Accumulates the parameter gradients into ``grads`` (dW1, db1, dW2, db2)
    and returns the gradient with respect to the MLP's input."""
    w1, _, w2, _ = p
    z, pre, hid = cache
    grads[2] += dy.T @ hid
    grads[3] += dy.sum(axis=0)
    dpre = (dy @ w2) * (pre > 0.0)
    grads[0] += dpre.T @ z
    grads[1] += dpre.sum(axis=0)
    return dpre @ w1


def _block_positions(n, rowptr, browptr, b):
    """Scalar CSR position of every entry of every b x b block, (nnzb, b, b),
    in the layout ``gnn.block_graph`` reads (the inverse of
    ``gnn.blocks_to_csr_values``)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    pos = np.empty((int(browptr[-1]), b, b), dtype=np.int64)
    for i in range(n // b):
        for q in range(browptr[i + 1] - browptr[i]):
            for r in range(b):
                base = rowptr[b * i + r] + b * q
                pos[browptr[i] + q, r] = base + np.arange(b)
    return pos


def gnn_forward_tape(n, rowptr, colidx, aval, node_feat, blob, n_layers=4, msg_raw_edge=False, b=1):
    """G values on A's pattern (as ``gnn.gnn_forward``, or for b > 1 as
    ``gnn.gnn_forward_blocks``: the GNN on the node graph of the b x b block
    matrix) and the tape the reverse pass reads."""
    aval = np.asarray(aval, dtype=np.float64)
    nrm = gnn.matrix_norm(aval)
    pos = None
    if b == 1:
        nodes, g_rowptr, g_colidx, eraw = n, rowptr, colidx, aval.reshape(-1, 1)
    else:
        nodes, g_rowptr, g_colidx, bval = gnn.block_graph(n, rowptr, colidx, aval, b)
        eraw = bval.reshape(-1, b * b)
        pos = _block_positions(n, rowptr, g_rowptr, b)
    node_feat = np.asarray(node_feat, dtype=np.float64).reshape(nodes, -1)
    d_node = node_feat.shape[1]
    params = gnn.unpack(blob, d_node, n_layers, msg_raw_edge, b)
    rows = np.repeat(np.arange(nodes), np.diff(np.asarray(g_rowptr, dtype=np.int64)))
    cols = np.asarray(g_colidx, dtype=np.int64)
    e = eraw / nrm
    n = nodes
    tape = {"n": n, "rows": rows, "cols": cols, "params": params, "d_node": d_node, "n_layers": n_layers,
            "msg_raw_edge": msg_raw_edge, "layers": [], "pos": pos, "b": b}
    x, tape["enc_n"] = _mlp_fwd(params[0], node_feat)
    h, tape["enc_e"] = _mlp_fwd(params[1], e)
    for t in range(n_layers):
        f_m, f_v, f_e = params[2 + 3 * t: 5 + 3 * t]
        edge_in = e if msg_raw_edge else h
        msg, c_m = _mlp_fwd(f_m, np.concatenate([x[rows], x[cols], edge_in], axis=1))
        m = np.zeros((n, gnn.HIDDEN))
        np.add.at(m, rows, msg)
        dx, c_v = _mlp_fwd(f_v, m)
        x = x + dx
        dh, c_e = _mlp_fwd(f_e, np.concatenate([x[rows], x[cols], h], axis=1))
        h = h + dh
        tape["layers"].append((c_m, c_v, c_e))
    g, tape["dec"] = _mlp_fwd(params[-1], h)
    if pos is None:
        return g[:, 0], tape
    out = np.empty(int(np.asarray(rowptr)[-1]))
    out[pos.reshape(-1)] = g.reshape(-1)
    return out, tape


def gnn_backward(tape, dg):
    """Gradient of a scalar objective with respect to the weight blob, given
    its gradient dg with respect to the G values (one per stored entry)."""
    n, rows, cols, params = tape["n"], tape["rows"], tape["cols"], tape["params"]
    d = gnn.HIDDEN
    grads = [[np.zeros_like(a) for a in p] for p in params]
    dg = np.asarray(dg, dtype=np.float64)
    if tape["pos"] is None:
        dy = dg.reshape(-1, 1)
    else:  # scalar CSR order -> one row of b^2 per block edge
        dy = dg[tape["pos"].reshape(len(tape["pos"]), -1)]
    dh = _mlp_bwd(params[-1], tape["dec"], dy, grads[-1])
    dx = np.zeros((n, d))
    for t in reversed(range(tape["n_layers"])):
        c_m, c_v, c_e = tape["layers"][t]
        i_m, i_v, i_e = 2 + 3 * t, 3 + 3 * t, 4 + 3 * t
        # h <- h + f_e(x_i, x_j, h), with x already updated
        dz = _mlp_bwd(params[i_e], c_e, dh, grads[i_e])
        np.add.at(dx, rows, dz[:, :d])
        np.add.at(dx, cols, dz[:, d:2 * d])
        dh = dh + dz[:, 2 * d:]
        # x <- x + f_v(m), m_i = sum over the row of f_m(x_i, x_j, edge)
        dm = _mlp_bwd(params[i_v], c_v, dx, grads[i_v])
        dz = _mlp_bwd(params[i_m], c_m, dm[rows], grads[i_m])
        np.add.at(dx, rows, dz[:, :d])
        np.add.at(dx, cols, dz[:, d:2 * d])
        if not tape["msg_raw_edge"]:
            dh = dh + dz[:, 2 * d:]
    _mlp_bwd(params[1], tape["enc_e"], dh, grads[1])
    _mlp_bwd(params[0], tape["enc_n"], dx, grads[0])
    out = []
    for w1, b1, w2, b2 in grads:
        out += [w1.ravel(), b1, w2.ravel(), b2]
    return np.concatenate(out)


def loss_and_grad(n, rowptr, colidx, aval, node_feat, blob, eps, w, n_layers=4, msg_raw_edge=False, b=1):
    """Mean SAI loss of the GNN's G (on A's full pattern; b x b blocks for
    b > 1) over the probes w, and its gradient with respect to the weight blob."""
    g, tape = gnn_forward_tape(n, rowptr, colidx, aval, node_feat, blob, n_layers, msg_raw_edge, b)
    loss, dg = sai_loss_grad_g(n, rowptr, colidx, aval, rowptr, colidx, g, eps, w)
    return loss, gnn_backward(tape, dg)
