"""Trains the GNN preconditioner on the GPU (Sec. 3.3 / Sec. 4.1).

The GNN of Sec. 3.2.2 (L = 4 message-passing layers, one hidden layer of 24
in every MLP) is trained on the SAI loss (Eqs. 7-8) with Hutchinson probes
w ~ N(0, 1), as the paper does: AdamW, batches of 4 matrices, an
exponentially decaying learning rate (x0.99 per epoch), eps = 1e-4 in
M^-1 = G G^T + eps I, a 4:1 train/test split.  Every step runs in libspai:
the forward pass (spai_gnn_precond), the loss and its gradient in G
(spai_sai_loss_grad), the reverse pass to the weights (spai_gnn_grad) and
the optimiser step (spai_adamw_step); this script only feeds them.

Data: the 3D variable-coefficient diffusion family (7-point finite volumes,
k = exp(sigma g), g a unit-variance Gaussian random field of correlation
length 8 cells; node features = position + log coefficient), at grid sides
12..24 with a seed per matrix -- small members of the family the solver is
benchmarked on (the GNN is local: 4 hops), standing in for the paper's heat
dataset, which is not available.  --sides and --sigmas widen it (a large
grid reaches larger |g| than a small one: at 128^3 k spans about e^+-8).

  python -m paper_2510_27517_gb300.train \\
      --out paper_2510_27517_gb300/weights/gnn_diffusion3d_l4

writes <out>.npy (the float32 weight blob, spai_gnn_weights layout) and
<out>.json (the configuration, the loss curve and the evaluation: PCG
iteration counts on the test matrices against random-init weights, Jacobi
and plain CG).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2510_27517_gb300 as spai  # noqa: E402
import workloads as W  # noqa: E402

D_NODE = 4  # node feature width; 1 with --features logk
LAYERS = 4


def node_features(k, features="pos_logk"):
    """Node features of a diffusion matrix: cell position in [-1, 1]^3 and
    log coefficient (d_node 4), or the log coefficient alone (d_node 1: the
    field is stationary, so position says nothing about the operator, and
    it means a different distance to the boundary on every grid size)."""
    f = W.diffusion3d_node_features(k)
    return np.ascontiguousarray(f[:, 3:4]) if features == "logk" else f


def dataset(count: int, sides, seed0: int, sigmas=(1.5,), features="pos_logk"):
    """`count` diffusion matrices, grid sides cycling through `sides` and
    field contrasts through `sigmas` (k = exp(sigma g)), each with its own
    random-field seed."""
    out = []
    for i in range(count):
        N = sides[i % len(sides)]
        sg = sigmas[(i // len(sides)) % len(sigmas)]
        A, k = W.diffusion3d(N, sg, 8.0, seed=seed0 + i)
        out.append({"N": N, "sigma": sg, "seed": seed0 + i, "A_h": A, "feat": node_features(k, features)})
    return out


def to_device(item):
    A_h = item["A_h"]
    A = spai.CSRMatrix.from_numpy(A_h.n, A_h.rowptr, A_h.colidx, A_h.val)
    item["A"] = A
    item["P"] = spai.build_pattern(A, spai.PATTERN_FULL)
    item["v"] = torch.tensor(item["feat"], device="cuda").contiguous()
    return item


def probes(n: int, k: int, seed: int) -> torch.Tensor:
    return torch.tensor(np.random.default_rng(seed).standard_normal((n, k)), device="cuda")


def loss_and_grad(item, blob: torch.Tensor, w: torch.Tensor, eps: float):
    M = spai.gnn_precond(item["A"], item["P"], item["v"], blob, d_node=D_NODE, n_layers=LAYERS, g_dtype=spai.F64,
                         eps=eps)
    loss, dG = spai.sai_loss_grad(item["A"], M, w)
    dW = spai.gnn_grad(item["A"], item["P"], item["v"], blob, dG, d_node=D_NODE, n_layers=LAYERS)
    M.close()
    return float(loss.mean().item()), dW


def mean_loss(items, blob, eps, k, seed):
    tot = 0.0
    for i, it in enumerate(items):
        M = spai.gnn_precond(it["A"], it["P"], it["v"], blob, d_node=D_NODE, n_layers=LAYERS, g_dtype=spai.F64,
                             eps=eps)
        tot += float(spai.sai_loss(it["A"], M, probes(it["A"].n, k, seed + i)).mean().item())
        M.close()
    return tot / len(items)


def pcg_iters(item, blob, eps, kind, max_iter=20000):
    """float64 PCG iterations to rtol 1e-8 with G from the GNN (`blob`),
    G = D^-1/2 (Jacobi) or G = I (plain CG)."""
    A, A_h = item["A"], item["A_h"]
    if kind == "gnn":
        M = spai.gnn_precond(A, item["P"], item["v"], blob, d_node=D_NODE, n_layers=LAYERS, g_dtype=spai.F64,
                             eps=eps)
    else:
        rows = np.repeat(np.arange(A_h.n), np.diff(A_h.rowptr))
        on = A_h.colidx == rows
        d = A_h.val[on][rows]
        g = np.where(on, 1.0 / np.sqrt(d) if kind == "jacobi" else 1.0, 0.0)
        M = spai.precond_from_values(item["P"], torch.tensor(g, device="cuda"), spai.F64, eps=0.0)
    b = torch.tensor(W.rhs_uniform(A_h.n, W.BASE_SEED + 10), device="cuda")
    x = torch.zeros(A_h.n, dtype=torch.float64, device="cuda")
    r = spai.pcg_solve(A, M, b, x, rtol=1e-8, max_iter=max_iter)
    M.close()
    return int(r["iters"]) if r["status"] == 0 else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--epochs", type=int, default=500)
    ap.add_argument("--matrices", type=int, default=40, help="matrices in the data set (4:1 train/test)")
    ap.add_argument("--sides", default="12,16,20,24")
    ap.add_argument("--sigmas", default="1.5",
                    help="field contrasts of the training matrices (large grids reach larger |g| than small ones)")
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--probes", type=int, default=8, help="Hutchinson probes per matrix and step")
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--decay", type=float, default=0.99, help="learning rate factor per epoch")
    ap.add_argument("--weight-decay", type=float, default=0.01)
    ap.add_argument("--clip", type=float, default=1.0, help="gradient 2-norm bound (0: none)")
    ap.add_argument("--eps", type=float, default=1e-4, help="shift of M^-1 = G G^T + eps I in training (the text's 1e-4)")
    ap.add_argument("--features", default="pos_logk", choices=["pos_logk", "logk"],
                    help="node features: position + log coefficient (d_node 4) or log coefficient alone (d_node 1)")
    ap.add_argument("--seed", type=int, default=W.BASE_SEED + 500)
    ap.add_argument("--eval-eps", type=float, default=1e-2, help="also evaluate with this shift")
    ap.add_argument("--eval-sides", default="48,64",
                    help="also count iterations on one matrix of each of these sides (sigma 1.5)")
    ap.add_argument("--eval-bench", type=int, default=1, help="also count iterations on the 128^3 benchmark matrix")
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2510_27517_gb300", "weights", "gnn_diffusion3d_l4"))
    args = ap.parse_args()

    global D_NODE
    D_NODE = 1 if args.features == "logk" else 4
    torch.cuda.set_device(0)
    spai.lib()
    sides = [int(s) for s in args.sides.split(",")]
    sigmas = [float(s) for s in args.sigmas.split(",")]
    data = [to_device(it) for it in dataset(args.matrices, sides, args.seed, sigmas, args.features)]
    n_test = max(1, args.matrices // 5)
    train, test = data[:-n_test], data[-n_test:]

    init = W.gnn_random_weights(D_NODE, LAYERS, seed=W.BASE_SEED + 100)
    init_desc = f"workloads.gnn_random_weights({D_NODE}, {LAYERS}, seed=BASE_SEED + 100)"
    blob = torch.tensor(init, device="cuda")
    master = blob.to(torch.float64).clone()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    g_acc = torch.zeros_like(master)
    rng = np.random.default_rng(args.seed + 1)
    curve = []
    step = 0
    t0 = time.time()
    test_loss0 = mean_loss(test, blob, args.eps, args.probes, 7)
    for epoch in range(args.epochs):
        lr = args.lr * args.decay ** epoch
        order = rng.permutation(len(train))
        ep_loss, ep_n = 0.0, 0
        for b0 in range(0, len(order), args.batch):
            idx = order[b0:b0 + args.batch]
            g_acc.zero_()
            for j in idx:
                it = train[j]
                w = probes(it["A"].n, args.probes, int(rng.integers(1 << 62)))
                loss, dW = loss_and_grad(it, blob, w, args.eps)
                g_acc += dW
                ep_loss += loss
                ep_n += 1
            g_acc /= len(idx)
            step += 1
            spai.adamw_step(master, m, v, g_acc, blob, step, lr, weight_decay=args.weight_decay,
                            max_grad_norm=args.clip)
        rec = {"epoch": epoch, "train_loss": ep_loss / ep_n, "lr": lr}
        if epoch % 25 == 0 or epoch == args.epochs - 1:
            rec["test_loss"] = mean_loss(test, blob, args.eps, args.probes, 7)
            print(json.dumps(rec), flush=True)
        curve.append(rec)
    train_s = time.time() - t0

    # evaluation: float64 PCG iterations to rtol 1e-8 on the test matrices
    evals = []
    init_blob = torch.tensor(init, device="cuda")
    extra = []
    for j, side in enumerate(int(x) for x in args.eval_sides.split(",") if x):
        extra += [to_device(it) for it in dataset(1, [side], args.seed + 10_000 + j, (1.5,), args.features)]
    if args.eval_bench:
        # the benchmark's own matrix (diffusion 128^3, sigma 1.5, its seed): evaluated, never trained on
        A, k = W.diffusion3d(128, 1.5, 8.0, seed=W.BASE_SEED + 2)
        extra.append(to_device({"N": 128, "sigma": 1.5, "seed": W.BASE_SEED + 2, "A_h": A,
                                "feat": node_features(k, args.features)}))
    for it in test + extra:
        evals.append({"N": it["N"], "sigma": it["sigma"], "seed": it["seed"], "n": it["A_h"].n,
                      "trained": pcg_iters(it, blob, args.eps, "gnn"),
                      "trained_eval_eps": pcg_iters(it, blob, args.eval_eps, "gnn"),
                      "random_init_eps0.3": pcg_iters(it, init_blob, 0.3, "gnn"),
                      "jacobi": pcg_iters(it, None, 0.0, "jacobi"),
                      "plain_cg": pcg_iters(it, None, 0.0, "identity")})
        print(json.dumps(evals[-1]), flush=True)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.save(args.out + ".npy", blob.cpu().numpy().astype(np.float32))
    meta = {"what": "GNN weight blob (spai_gnn_weights layout, float32) trained on the SAI loss",
            "d_node": D_NODE, "n_layers": LAYERS, "msg_edge": "latent", "block": 1, "eps": args.eps,
            "count": int(blob.numel()),
            "data": {"family": "diffusion3d (7-point FV, k = exp(1.5 g), correlation length 8 cells)",
                     "sides": sides, "sigmas": sigmas, "matrices": args.matrices, "train": len(train),
                     "test": len(test),
                     "seed0": args.seed},
            "optimiser": {"kind": "AdamW", "lr": args.lr, "decay_per_epoch": args.decay,
                          "weight_decay": args.weight_decay, "clip": args.clip, "batch": args.batch,
                          "probes": args.probes, "epochs": args.epochs, "steps": step},
            "init": init_desc, "features": args.features,
            "test_loss_init": test_loss0, "test_loss_final": curve[-1].get("test_loss"),
            "train_seconds": train_s, "curve": [c for c in curve if "test_loss" in c],
            "eval_pcg_f64_rtol1e-8": evals,
            "command": "python -m paper_2510_27517_gb300.train " + " ".join(sys.argv[1:])}
    with open(args.out + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps({"done": True, "train_seconds": train_s, "test_loss_init": test_loss0,
                      "test_loss_final": curve[-1].get("test_loss")}))


if __name__ == "__main__":
    main()
