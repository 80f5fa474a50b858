"""Neighbourhood extraction for checking the GNN at full size on sampled rows.

After L message-passing layers (Eq. 4) the value G_ij depends only on the
nodes within L + 1 hops of i: x_j^(L) needs x^(L-1) one hop further out, down
to x^(0) at distance L + 1, and the aggregation at a node is complete as long
as all its neighbours are inside the ball.  So G on the rows of a seed set
is reproduced exactly by the forward pass on the (L + 1)-hop ball around the
seeds, with the edge features scaled by the norm of the whole matrix."""
from __future__ import annotations

import numpy as np

import workloads as W


def ball(A: W.CSR, seeds, radius: int):
    """Sorted node list of the radius-hop neighbourhood of `seeds`."""
    n = A.n
    mark = np.zeros(n, dtype=bool)
    front = np.unique(np.asarray(seeds, dtype=np.int64))
    mark[front] = True
    rp = A.rowptr.astype(np.int64)
    for _ in range(radius):
        if front.size == 0:
            break
        starts, ends = rp[front], rp[front + 1]
        idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)])
        nb = np.unique(A.colidx[idx].astype(np.int64))
        nb = nb[~mark[nb]]
        mark[nb] = True
        front = nb
    return np.nonzero(mark)[0]


def submatrix(A: W.CSR, nodes: np.ndarray):
    """A restricted to `nodes` (sorted), columns relabelled monotonically so
    every row keeps its stored order.  Returns the sub-CSR and, for every
    stored entry of the sub-matrix, its entry index in A."""
    n = A.n
    local = np.full(n, -1, dtype=np.int64)
    local[nodes] = np.arange(nodes.size)
    rp = A.rowptr.astype(np.int64)
    ent = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in nodes])
    rows = np.repeat(np.arange(nodes.size), rp[nodes + 1] - rp[nodes])
    cols = local[A.colidx[ent].astype(np.int64)]
    keep = cols >= 0
    ent, rows, cols = ent[keep], rows[keep], cols[keep]
    rowptr = np.zeros(nodes.size + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    sub = W.CSR(nodes.size, rowptr.astype(np.int32), cols.astype(np.int32), np.asarray(A.val)[ent])
    return sub, ent


def entries_of_rows(A: W.CSR, rows) -> np.ndarray:
    rp = A.rowptr.astype(np.int64)
    return np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
