"""Build GNN weight blobs from sparse hand-set entries (test helper)."""
import numpy as np

from workloads import HIDDEN, gnn_layer_shapes


def blob_from_entries(d_node, n_layers, entries, msg_raw_edge=False):
    shapes = gnn_layer_shapes(d_node, n_layers, msg_raw_edge)
    offs = {}
    o = 0
    for name, fi, fo in shapes:
        offs[name] = {"W1": (o, (HIDDEN, fi)), "b1": (o + HIDDEN * fi, (HIDDEN,)),
                      "W2": (o + HIDDEN * fi + HIDDEN, (fo, HIDDEN)),
                      "b2": (o + HIDDEN * fi + HIDDEN + fo * HIDDEN, (fo,))}
        o += HIDDEN * fi + HIDDEN + fo * HIDDEN + fo
    blob = np.zeros(o, dtype=np.float32)
    for name, part, idx, val in entries:
        base, shape = offs[name][part]
        flat = np.ravel_multi_index(tuple(idx), shape)
        blob[base + flat] = val
    return blob, offs
