"""GNN forward pass that writes the values of G (oracle).

Follows Sec. 3.2.2 of the paper, Eqs. 3-5, in float64:

* matrix norm (Sec. 3.3): ||A|| = mean over stored entries of |A_ij|;
  the edge feature is e_ij = A_ij / ||A|| (d_edge = 1, block size b = 1);
* encoder (Eq. 3): x_i = E_n(v_i), h_ij = E_e(e_ij);
* L message-passing layers (Eq. 4), for t = 1..L:
    m_i  = sum over j in N(i) of f_m(x_i, x_j, h_ij)
    x_i <- x_i + f_v(m_i)
    h_ij <- h_ij + f_e(x_i, x_j, h_ij)      (x already updated)
* decoder (Eq. 5): G_ij = D(h_ij), written on A's pattern.

N(i) is every stored entry of row i, the diagonal included (the graph of A
has an edge wherever A_ij != 0, Sec. 3.1).

Readings of points the paper leaves open (Sec. 4.1 fixes only L = 4, one
hidden layer of width 24 per MLP and about 24k parameters):
* every MLP is Linear(fan_in -> 24), ReLU, Linear(24 -> fan_out);
* f_m and f_e take the concatenation (x_i, x_j, edge) in that order, f_v takes
  m_i only;
* the message's edge input is the current latent h_ij (default) or, with
  ``msg_raw_edge=True``, the raw feature e_ij exactly as Eq. 4 prints it.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 24


def layer_shapes(d_node: int, n_layers: int, msg_raw_edge: bool = False, b: int = 1):
    """(fan_in, fan_out) per MLP in blob order: E_n, E_e, (f_m, f_v, f_e) x L, D.
    With b x b blocks the edge feature and the decoder output have b^2 entries."""
    d = HIDDEN
    d_edge = b * b
    shapes = [(d_node, d), (d_edge, d)]
    for _ in range(n_layers):
        shapes += [(2 * d + (d_edge if msg_raw_edge else d), d), (d, d), (3 * d, d)]
    shapes.append((d, b * b))
    return shapes


def unpack(blob: np.ndarray, d_node: int, n_layers: int, msg_raw_edge: bool = False, b: int = 1):
    """Split the flat blob into [(W1, b1, W2, b2)] per MLP, float64.
    Layout per MLP: W1 (24 x fan_in, row-major), b1 (24), W2 (fan_out x 24), b2."""
    blob = np.asarray(blob, dtype=np.float64)
    out, o = [], 0
    for fi, fo in layer_shapes(d_node, n_layers, msg_raw_edge, b):
        w1 = blob[o:o + HIDDEN * fi].reshape(HIDDEN, fi); o += HIDDEN * fi
        b1 = blob[o:o + HIDDEN]; o += HIDDEN
        w2 = blob[o:o + fo * HIDDEN].reshape(fo, HIDDEN); o += fo * HIDDEN
        b2 = blob[o:o + fo]; o += fo
        out.append((w1, b1, w2, b2))
    if o != blob.shape[0]:
        raise ValueError(f"weight blob has {blob.shape[0]} values, layout needs {o}")
    return out


def mlp(p, z: np.ndarray) -> np.ndarray:
    """One hidden layer: W2 relu(W1 z + b1) + b2, applied to each row of z."""
    w1, b1, w2, b2 = p
    hid = np.maximum(z @ w1.T + b1, 0.0)
    return hid @ w2.T + b2


def matrix_norm(aval: np.ndarray) -> float:
    """Dimension-agnostic norm of Sec. 3.3: mean of |A_ij| over stored entries."""
    return float(np.mean(np.abs(np.asarray(aval, dtype=np.float64))))


def gnn_forward(n: int, rowptr: np.ndarray, colidx: np.ndarray, aval: np.ndarray,
                node_feat: np.ndarray, blob: np.ndarray, n_layers: int = 4,
                msg_raw_edge: bool = False, return_latents: bool = False, a_norm: float | None = None):
    """Values of G on A's pattern (one per stored entry, CSR order).

    ``a_norm`` is ||A|| (Sec. 3.3) when the given rows are a sub-block of a
    larger matrix whose own norm must scale the edge features; by default
    it is computed from ``aval``."""
    g, x, h = _forward(n, rowptr, colidx, np.asarray(aval, dtype=np.float64).reshape(-1, 1), node_feat, blob,
                       n_layers, msg_raw_edge, 1, matrix_norm(aval) if a_norm is None else float(a_norm))
    g = g[:, 0]
    if return_latents:
        return g, x, h
    return g


def block_graph(n: int, rowptr, colidx, val, b: int):
    """The node graph of a scalar CSR made of dense b x b blocks (each block
    row's b scalar rows list the same blocks in column order, b entries per
    block): (nb, block rowptr, block columns, block values (nnzb, b, b))."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colidx = np.asarray(colidx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    if n % b:
        raise ValueError("n is not a multiple of the block size")
    nb = n // b
    lens = np.diff(rowptr).reshape(nb, b)
    if np.any(lens != lens[:, :1]) or np.any(lens % b):
        raise ValueError("rows of a block row differ or are not whole blocks")
    bl = lens[:, 0] // b
    browptr = np.concatenate([[0], np.cumsum(bl)])
    nnzb = int(browptr[-1])
    bcol = np.empty(nnzb, dtype=np.int64)
    bval = np.empty((nnzb, b, b))
    for i in range(nb):
        for q in range(bl[i]):
            k = browptr[i] + q
            for r in range(b):
                base = rowptr[b * i + r] + b * q
                cols = colidx[base:base + b]
                if cols[0] % b or np.any(cols != cols[0] + np.arange(b)):
                    raise ValueError("columns do not form aligned blocks")
                if r == 0:
                    bcol[k] = cols[0] // b
                elif cols[0] // b != bcol[k]:
                    raise ValueError("rows of a block row list different blocks")
                bval[k, r] = val[base:base + b]
    return nb, browptr, bcol, bval


def blocks_to_csr_values(n: int, rowptr, browptr, gblocks, b: int) -> np.ndarray:
    """Values of b x b blocks in the scalar CSR order of ``block_graph``'s input."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    out = np.empty(int(rowptr[-1]))
    for i in range(n // b):
        for q in range(browptr[i + 1] - browptr[i]):
            for r in range(b):
                base = rowptr[b * i + r] + b * q
                out[base:base + b] = gblocks[browptr[i] + q, r]
    return out


def gnn_forward_blocks(n: int, rowptr, colidx, aval, node_feat, blob, b: int, n_layers: int = 4,
                       msg_raw_edge: bool = False) -> np.ndarray:
    """Block version (the paper's b x b blocks, Sec. 3.2.2 with d_edge = b^2):
    the GNN runs on the node graph of the block matrix, every edge feature is
    the block of A / ||A|| flattened row-major (||A|| over all stored scalar
    entries), and the decoder writes a b x b block of G per edge.  Input and
    output are in the scalar CSR of A (dense blocks)."""
    nb, browptr, bcol, bval = block_graph(n, rowptr, colidx, aval, b)
    e = bval.reshape(-1, b * b)
    g, _, _ = _forward(nb, browptr, bcol, e, node_feat, blob, n_layers, msg_raw_edge, b, matrix_norm(aval))
    return blocks_to_csr_values(n, rowptr, browptr, g.reshape(-1, b, b), b)


def _forward(n, rowptr, colidx, eraw, node_feat, blob, n_layers, msg_raw_edge, b, nrm):
    """Eqs. 3-5 on a graph with n nodes; eraw: raw edge features (nnz, b^2)."""
    node_feat = np.asarray(node_feat, dtype=np.float64).reshape(n, -1)
    d_node = node_feat.shape[1]
    params = unpack(blob, d_node, n_layers, msg_raw_edge, b)
    E_n, E_e, D = params[0], params[1], params[-1]
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    cols = np.asarray(colidx, dtype=np.int64)
    e = eraw / nrm

    x = mlp(E_n, node_feat)
    h = mlp(E_e, e)
    for t in range(n_layers):
        f_m, f_v, f_e = params[2 + 3 * t: 5 + 3 * t]
        edge_in = e if msg_raw_edge else h
        msg = mlp(f_m, np.concatenate([x[rows], x[cols], edge_in], axis=1))
        m = np.zeros((n, HIDDEN))
        np.add.at(m, rows, msg)          # sum over j in N(i)
        x = x + mlp(f_v, m)
        h = h + mlp(f_e, np.concatenate([x[rows], x[cols], h], axis=1))
    return mlp(D, h), x, h
