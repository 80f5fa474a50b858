"""PCG on the GPU against the oracle's Algorithm 1 (App. A) with
M^-1 = G G^T + eps I (Eq. 1).

float64 path: per-iteration residual norms agree to 1e-10 relative and x to
1e-8 relative (same iteration, same G).  Special cases G = I and
G = D^-1/2.  Mixed precision: the true float64 residual reaches rtol."""
import numpy as np
import pytest
import torch

import paper_2510_27517_gb300 as spai_mod
import workloads as W
from oracle import fsai, pcg

pytestmark = pytest.mark.gpu


def assert_history_parity(hist, ref_hist, bnorm):
    """Per-iteration ||r_k|| parity.  Differences in dot-product summation
    order are amplified by CG roughly as eps * ||r_0|| / ||r_k||, so the
    1e-10 bar is taken relative to ||b|| (the scale of rtol) at every
    iteration, and relative to ||r_k|| itself while ||r_k|| >= 1e-4 ||b||."""
    ref_hist = np.asarray(ref_hist)
    assert hist.shape == ref_hist.shape
    diff = np.abs(hist - ref_hist)
    assert (diff / bnorm).max() <= 1e-10, (diff / bnorm).max()
    early = ref_hist >= 1e-4 * bnorm
    assert (diff[early] / ref_hist[early]).max() <= 1e-10, (diff[early] / ref_hist[early]).max()


def stable_window(A, b, apply, ref, tol=1e-11):
    """Iterations over which the oracle agrees with itself when every apply
    is perturbed by about one rounding (relative 1e-16): the horizon up to
    which per-iteration parity is a property of the method at all."""
    rng = np.random.default_rng(0)
    alt = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, lambda r: apply(r) * (1 + 1e-16 * rng.standard_normal(A.n)),
                  rtol=1e-8)
    m = min(len(ref.history), len(alt.history))
    d = np.abs(np.asarray(ref.history[:m]) - np.asarray(alt.history[:m])) / np.linalg.norm(b)
    bad = np.nonzero(d > tol)[0]
    return int(bad[0]) if bad.size else m


def upload(spai, A):
    return spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)


def fsai_precond(spai, A, dA, g_dtype=0):
    urp, uci, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
    pat = spai.build_pattern(dA, spai.PATTERN_UPPER)
    return spai.precond_from_values(pat, torch.tensor(gv, device="cuda"), g_dtype, eps=0.0), (urp, uci, gv)


def gpu_solve(spai, dA, M, b, hist_len=0, **kw):
    x = torch.zeros(dA.n, dtype=torch.float64, device="cuda")
    h = torch.zeros(hist_len, dtype=torch.float64, device="cuda") if hist_len else None
    res = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, history=h, **kw)
    return res, x.cpu().numpy(), (h.cpu().numpy() if h is not None else None)


def test_poisson64_fsai_matches_oracle_every_iteration(spai_lib):
    spai = spai_lib
    A = W.poisson2d(64)
    b = W.rhs_uniform(A.n, W.BASE_SEED + 1)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-8)
    res, x, hist = gpu_solve(spai, dA, M, b, hist_len=4096)
    assert res["status"] == 0 and ref.status == pcg.CONVERGED
    assert res["iters"] == ref.iters
    k = res["history_written"]
    assert k == len(ref.history)
    assert_history_parity(hist[:k], ref.history, np.linalg.norm(b))
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    assert res["true_rel_res"] <= 1e-8
    assert abs(res["true_rel_res"] - pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x, b)) < 1e-12


@pytest.mark.parametrize("which", ["identity", "jacobi"])
@pytest.mark.parametrize("period", [50, 0, 7])
def test_special_cases(spai_lib, which, period):
    spai = spai_lib
    A = W.aniso2d(23, 40.0, 0.6)
    b = W.rhs_uniform(A.n, 11)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.val[A.colidx == rows]
    g = np.where(A.colidx == rows, 1.0 if which == "identity" else 1.0 / np.sqrt(diag[rows]), 0.0)
    dA = upload(spai, A)
    pat = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.precond_from_values(pat, torch.tensor(g, device="cuda"), spai.F64, eps=0.0)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g, 0.0),
                  rtol=1e-9, replace_period=period)
    res, x, hist = gpu_solve(spai, dA, M, b, hist_len=8192, rtol=1e-9, replace_period=period)
    assert res["iters"] == ref.iters
    k = res["history_written"]
    assert_history_parity(hist[:k], ref.history, np.linalg.norm(b))
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_precond_criterion(spai_lib):
    spai = spai_lib
    A = W.poisson2d(30)
    b = W.rhs_uniform(A.n, 3)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-8,
                  criterion=pcg.PRECOND)
    res, x, _ = gpu_solve(spai, dA, M, b, criterion=spai.CRIT_PRECOND)
    assert res["iters"] == ref.iters and res["status"] == 0
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_zero_rhs_and_not_converged(spai_lib):
    spai = spai_lib
    A = W.poisson2d(16)
    dA = upload(spai, A)
    M, _ = fsai_precond(spai, A, dA)
    res, x, _ = gpu_solve(spai, dA, M, np.zeros(A.n))
    assert res["status"] == 0 and res["iters"] == 0 and not x.any()
    res, x, _ = gpu_solve(spai, dA, M, W.rhs_uniform(A.n, 1), max_iter=5)
    assert res["status"] == spai.spai.ERR_NOT_CONVERGED and res["iters"] == 5
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, W.rhs_uniform(A.n, 1),
                  pcg.spai_apply(A.n, *fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val), 0.0), max_iter=5)
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


def test_nonzero_x0(spai_lib):
    spai = spai_lib
    A = W.poisson2d(24)
    b = W.rhs_uniform(A.n, 5)
    x0 = W.rhs_uniform(A.n, 6)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), x0=x0)
    x = torch.tensor(x0, device="cuda")
    res = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x)
    assert res["iters"] == ref.iters
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("gdt", [1, 2, 3])
def test_mixed_precision_reaches_rtol(spai_lib, gdt):
    spai = spai_lib
    A = W.poisson2d(64)
    b = W.rhs_uniform(A.n, W.BASE_SEED + 1)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA, g_dtype=gdt)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-8)
    res, x, _ = gpu_solve(spai, dA, M, b, precision=spai.PREC_MIXED)
    assert res["status"] == 0
    true = pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x, b)
    assert true <= 1e-8 and abs(true - res["true_rel_res"]) < 1e-12
    # the distance to the oracle's x is bounded by the conditioning of A times rtol
    assert np.linalg.norm(x - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_mixed_first_inner_solve_tracks_oracle(spai_lib):
    # first inner float32 iterations follow the float64 oracle on the same data
    spai = spai_lib
    A = W.poisson2d(40)
    b = W.rhs_uniform(A.n, 2)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA, g_dtype=1)
    a32 = A.val.astype(np.float32).astype(np.float64)
    g32 = gv.astype(np.float32).astype(np.float64)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, a32, b.astype(np.float32).astype(np.float64),
                  pcg.spai_apply(A.n, urp, uci, g32, 0.0), rtol=1e-4)
    res, x, hist = gpu_solve(spai, dA, M, b, hist_len=4096, precision=spai.PREC_MIXED, inner_rtol=1e-4)
    k = min(20, len(ref.history))
    rel = np.abs(hist[:k] - np.array(ref.history[:k])) / np.array(ref.history[:k])
    assert rel.max() <= 1e-4, rel


def test_batched_equals_alone(spai_lib):
    spai = spai_lib
    mats = [W.poisson2d(20), W.aniso2d(31, 10.0, 0.3), W.poisson2d(45), W.aniso2d(12, 500.0, 2.0)]
    systems, preconds, bs, xs = [], [], [], []
    alone = []
    for i, A in enumerate(mats):
        dA = upload(spai, A)
        S = spai.system_create(dA)
        M, _ = fsai_precond(spai, A, dA)
        b = torch.tensor(W.rhs_uniform(A.n, 100 + i), device="cuda")
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = spai.system_solve(S, M, b, x)
        alone.append((r, x.clone()))
        systems.append(S); preconds.append(M); bs.append(b)
        xs.append(torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    res = spai.pcg_solve_batched(systems, preconds, bs, xs)
    for (ra, xa), rb, xb in zip(alone, res, xs):
        assert rb["status"] == 0 and rb["iters"] == ra["iters"]
        assert torch.equal(xa, xb)


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_over_many_rounds_equals_alone(spai_lib, mixed):
    # one work item per row group (items_log2 -4): the batch holds several
    # times more items than the grid has blocks, so every block runs items of
    # several members per pass, dealt by size in a snake, and members that
    # finish early are dealt out between launches; each member's iteration
    # is bit-identical to its solve alone (where its own items take more than
    # one round too)
    spai = spai_lib
    gdt = spai.F32 if mixed else spai.F64
    prec = spai.PREC_MIXED if mixed else spai.PREC_F64
    mats = [W.aniso2d(300, 30.0, 0.4), W.poisson2d(60), W.aniso2d(220, 5.0, 1.1), W.poisson2d(150),
            W.aniso2d(40, 200.0, 2.5), W.aniso2d(180, 2.0, 0.2)]
    blob = torch.tensor(W.gnn_random_weights(1, 4), device="cuda")
    systems, preconds, bs, keep, alone = [], [], [], [], []
    for i, A in enumerate(mats):
        dA = upload(spai, A)
        S = spai.system_create(dA)
        S.set_schedule(items_log2=-4)
        P = spai.build_pattern(dA, spai.PATTERN_FULL)
        M = spai.gnn_precond(dA, P, torch.tensor(W.row_average_feature(A), device="cuda"), blob, d_node=1,
                             g_dtype=gdt, eps=0.3)
        b = torch.tensor(W.rhs_uniform(A.n, 300 + i), device="cuda")
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        alone.append((spai.system_solve(S, M, b, x, precision=prec), x.clone()))
        systems.append(S), preconds.append(M), bs.append(b), keep.append((dA, P))
    xs = [torch.zeros_like(b) for b in bs]
    res = spai.pcg_solve_batched(systems, preconds, bs, xs, precision=prec)
    iters = [r["iters"] for r in res]
    assert max(iters) > 2 * min(iters)  # members finish at different times
    for (ra, xa), rb, xb in zip(alone, res, xs):
        assert rb["status"] == 0 and ra["status"] == 0
        assert rb["iters"] == ra["iters"] and rb["outer_iters"] == ra["outer_iters"]
        assert torch.equal(xa, xb)


@pytest.mark.parametrize("mixed", [False, True])
def test_sell_and_csr_members_in_one_launch(spai_lib, mixed):
    # a launch whose members all stream SELL-32 slices runs the kernel built
    # without the CSR ring; a batch that also holds a CSR system runs the full
    # kernel: each member's iteration is bit-identical either way
    spai = spai_lib
    gdt = spai.F32 if mixed else spai.F64
    prec = spai.PREC_MIXED if mixed else spai.PREC_F64
    A1, k1 = W.diffusion3d(14)
    d1 = upload(spai, A1)
    S1 = spai.system_create(d1)
    assert S1.schedule()["sell"] == 1
    P1 = spai.build_pattern(d1, spai.PATTERN_FULL)
    M1 = spai.gnn_precond(d1, P1, torch.tensor(W.diffusion3d_node_features(k1), device="cuda"),
                          torch.tensor(W.gnn_random_weights(4, 4), device="cuda"), d_node=4, g_dtype=gdt, eps=0.3)
    A2 = W.aniso2d(40, 20.0, 0.7)
    d2 = upload(spai, A2)
    S2 = spai.system_create(d2)
    S2.set_schedule(sell=0, staged=1)  # CSR row groups through the stage ring
    M2, _ = fsai_precond(spai, A2, d2, gdt)
    bs = [torch.tensor(W.rhs_uniform(A1.n, 41), device="cuda"), torch.tensor(W.rhs_uniform(A2.n, 42), device="cuda")]
    alone = []
    for S, M, b in ((S1, M1, bs[0]), (S2, M2, bs[1])):
        x = torch.zeros(b.numel(), dtype=torch.float64, device="cuda")
        r = spai.system_solve(S, M, b, x, precision=prec)
        assert r["status"] == 0
        alone.append((r, x))
    xs = [torch.zeros_like(alone[0][1]), torch.zeros_like(alone[1][1])]
    res = spai.pcg_solve_batched([S1, S2], [M1, M2], bs, xs, precision=prec)
    for (ra, xa), rb, xb in zip(alone, res, xs):
        assert rb["status"] == 0 and rb["iters"] == ra["iters"] and rb["outer_iters"] == ra["outer_iters"]
        assert torch.equal(xa, xb)


def test_mixed_reliable_updates_track_f64_iteration_count(spai_lib):
    # float32 iterations with float64 refinement of x and r reach the float64
    # rtol in about the float64 iteration count (the recurrence is not restarted)
    spai = spai_lib
    A = W.aniso2d(90, 300.0, 0.4)
    b = W.rhs_uniform(A.n, 9)
    dA = upload(spai, A)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.val[A.colidx == rows]
    g = np.where(A.colidx == rows, 1.0 / np.sqrt(diag[rows]), 0.0)
    pat = spai.build_pattern(dA, spai.PATTERN_FULL)
    M64 = spai.precond_from_values(pat, torch.tensor(g, device="cuda"), spai.F64, eps=0.0)
    M32 = spai.precond_from_values(pat, torch.tensor(g, device="cuda"), spai.F32, eps=0.0)
    r64, x64, _ = gpu_solve(spai, dA, M64, b)
    r32, x32, _ = gpu_solve(spai, dA, M32, b, precision=spai.PREC_MIXED)
    assert r64["status"] == 0 and r32["status"] == 0
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x32, b) <= 1e-8
    assert r32["iters"] <= 1.3 * r64["iters"] + 10, (r32["iters"], r64["iters"])
    assert r32["outer_iters"] >= 1


def test_autotuned_schedule_fixed_and_batch_consistent(spai_lib):
    # the first solve of an autotuned system picks its schedule by timing;
    # afterwards the schedule is fixed: the same result alone and in a batch
    spai = spai_lib
    A = W.aniso2d(150, 50.0, 0.9)
    dA = upload(spai, A)
    S = spai.system_create(dA, autotune=True)
    assert S.schedule()["tuned"] == 0
    M, _ = fsai_precond(spai, A, dA)
    b = torch.tensor(W.rhs_uniform(A.n, 21), device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r1 = spai.system_solve(S, M, b, x)
    sch = S.schedule()
    assert sch["tuned"] == 1 and sch["tile_nnz"] >= 256 and sch["items_log2"] in (-1, 0, 1)
    assert r1["status"] == 0
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.cpu().numpy(), b.cpu().numpy()) <= 1e-8
    x2 = torch.zeros_like(x)
    r2 = spai.system_solve(S, M, b, x2)
    assert S.schedule() == sch and r2["iters"] == r1["iters"] and torch.equal(x, x2)
    B = W.poisson2d(40)
    dB = upload(spai, B)
    SB = spai.system_create(dB)
    MB, _ = fsai_precond(spai, B, dB)
    bB = torch.tensor(W.rhs_uniform(B.n, 22), device="cuda")
    xs = [torch.zeros_like(x), torch.zeros(B.n, dtype=torch.float64, device="cuda")]
    res = spai.pcg_solve_batched([S, SB], [M, MB], [b, bB], xs)
    assert res[0]["iters"] == r1["iters"] and torch.equal(xs[0], x)
    assert res[1]["status"] == 0


@pytest.mark.parametrize("sched", [dict(sell=1), dict(sell=0, staged=1), dict(sell=0, staged=0),
                                   dict(sell=1, tile_nnz=300, items_log2=2), dict(sell=0, tile_nnz=257, items_log2=-2),
                                   dict(sell=1, fuse=0), dict(sell=0, staged=0, fuse=0),
                                   dict(matrix="graph", sell=1), dict(matrix="graph", sell=1, fuse=0),
                                   dict(matrix="graph", sell=1, tile_nnz=300, items_log2=1),
                                   dict(matrix="graph", sell=0, staged=1), dict(matrix="graph", sell=1, pair=0),
                                   dict(sell=1, pair=1), dict(sell=0, staged=1, pair=1)])
def test_every_schedule_matches_oracle(spai_lib, sched):
    # SELL-32 slices (rows in their own order for the stencil; ordered by
    # length within windows for the graph Laplacian, whose rows are too
    # uneven for plain slices) and CSR row groups (staged or direct), any
    # group size: the same float64 iteration as the oracle's Algorithm 1
    spai = spai_lib
    sched = dict(sched)
    graph = sched.pop("matrix", "stencil") == "graph"
    if graph:
        A = W.graph_laplacian(3000, 24000, seed=13)
        v, d_node = W.row_average_feature(A), 1
    else:
        A, k = W.diffusion3d(12)
        v, d_node = W.diffusion3d_node_features(k), 4
    dA = upload(spai, A)
    S = spai.system_create(dA)
    lay = S.layout()
    assert lay["sell_slices"] > 0 and lay["sell_sorted"] == (1 if graph else 0)
    assert lay["sell_total"] * 4 <= A.nnz * 5
    assert S.schedule()["pair"] == (1 if graph else 0)  # paired vectors by default for sorted rows
    S.set_schedule(**sched)
    assert S.schedule()["tuned"] == 1
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"),
                         torch.tensor(W.gnn_random_weights(d_node, 4), device="cuda"), d_node=d_node,
                         g_dtype=spai.F64, eps=0.3)
    g, _ = M.export(spai.F64)
    b = W.rhs_uniform(A.n, 31)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g.cpu().numpy(), 0.3),
                  rtol=1e-8)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    h = torch.zeros(20000, dtype=torch.float64, device="cuda")
    r = spai.system_solve(S, M, torch.tensor(b, device="cuda"), x, history=h)
    assert r["status"] == 0 and abs(r["iters"] - ref.iters) <= 0.03 * ref.iters + 1
    # with a random-weight G this iteration is chaotic: two oracle runs whose
    # applies differ by one rounding part company after a few dozen steps, so
    # the per-iteration bar holds over the window where they still agree
    k0 = stable_window(A, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g.cpu().numpy(), 0.3), ref)
    assert k0 >= 10
    assert_history_parity(h[:k0].cpu().numpy(), ref.history[:k0], np.linalg.norm(b))
    xh = x.cpu().numpy()
    assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, xh, b) <= 1e-8
    assert np.linalg.norm(xh - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_set_schedule_rejects_out_of_range(spai_lib):
    spai = spai_lib
    A = W.poisson2d(16)
    S = spai.system_create(upload(spai, A))
    for bad in (dict(tile_nnz=5000), dict(items_log2=5), dict(staged=2), dict(sell=-1), dict(fuse=2), dict(pair=2)):
        with pytest.raises(spai.SpaiError):
            S.set_schedule(**bad)


def test_lanczos_coefficients_and_condition_estimates(spai_lib):
    # the solve's alpha / beta against the oracle's, and the Ritz estimates of
    # kappa and Kaporin's number (Sec. 4.5) against the dense spectrum
    from oracle import spectrum
    spai = spai_lib
    A = W.poisson2d(32)
    b = W.rhs_uniform(A.n, 41)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-10)
    lz = torch.zeros(2 * 4096, dtype=torch.float64, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = spai.pcg_solve(dA, M, torch.tensor(b, device="cuda"), x, rtol=1e-10, lanczos=lz)
    k = r["lanczos_written"]
    assert r["status"] == 0 and k == r["iters"] == ref.iters == len(ref.alphas)
    al = lz[0::2][:k].cpu().numpy()
    be = lz[1::2][:k - 1].cpu().numpy()
    assert np.allclose(al, ref.alphas, rtol=1e-9)
    assert np.allclose(be, ref.betas[:k - 1], rtol=1e-9)
    lam = spectrum.preconditioned_eigenvalues(A.n, A.rowptr, A.colidx, A.val, urp, uci, gv, 0.0)
    lo, hi = spai.ritz_extremes(al, be)
    assert lo >= lam[0] * (1 - 1e-9) and hi <= lam[-1] * (1 + 1e-9)
    assert hi / lo == pytest.approx(spectrum.kappa(lam), rel=1e-2)
    ritz_o = spectrum.ritz_values(ref.alphas, ref.betas[:k - 1])
    assert hi / lo == pytest.approx(ritz_o.max() / ritz_o.min(), rel=1e-8)
    kap = spai.ritz_kaporin(al, be)
    assert 1.0 < kap < hi / lo
    assert kap == pytest.approx(spectrum.kappa_kaporin(lam), rel=0.25)


def test_bounded_waits_time_out_and_context_survives(spai_lib):
    # a grid barrier nobody releases and an mbarrier nothing arrives on give up
    # after 20 ms with a timeout status; a solve afterwards still works
    spai = spai_lib
    assert spai.selftest_wait_timeout(20000)
    A = W.poisson2d(16)
    dA = upload(spai, A)
    M, _ = fsai_precond(spai, A, dA)
    res, x, _ = gpu_solve(spai, dA, M, W.rhs_uniform(A.n, 3))
    assert res["status"] == 0


def test_host_buffer_solve_poisson64(spai_lib):
    # spai_pcg_solve_host: b and x in (pinned) host memory, the copies inside
    # the call; the 64 x 64 Poisson FSAI solve against the oracle
    spai = spai_lib
    A = W.poisson2d(64)
    b = W.rhs_uniform(A.n, W.BASE_SEED + 1)
    dA = upload(spai, A)
    M, (urp, uci, gv) = fsai_precond(spai, A, dA)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, urp, uci, gv, 0.0), rtol=1e-8)
    for pinned in (True, False):
        b_h = torch.tensor(b)
        x_h = torch.zeros(A.n, dtype=torch.float64)
        if pinned:
            b_h, x_h = b_h.pin_memory(), x_h.pin_memory()
        res = spai.pcg_solve_host(dA, M, b_h, x_h)
        assert res["status"] == 0 and res["iters"] == ref.iters
        x = x_h.numpy()
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x, b) <= 1e-8


@pytest.mark.parametrize("flag", ["fuse", "pair"])
@pytest.mark.parametrize("case", ["gnn_sell_mixed", "gnn_csr_f64", "fsai_upper", "graph_direct", "graph_sell",
                                  "batch"])
def test_schedule_flags_are_bit_identical(spai_lib, case, flag):
    # fuse: the G^T and G passes in one grid step, ordered by item flags, run
    # the same arithmetic as one grid step per pass.  pair: s with d and q
    # with r stored as interleaved pairs (one load per gathered pair) run the
    # same arithmetic as separate vectors.  Identical iterates, residual
    # histories and iteration counts, for SELL-32 (rows in order and sorted by
    # length) and CSR (staged and direct) layouts, a factor whose G and G^T
    # have different row structure (FSAI on the upper triangle) and a batch
    # (pair: only every other member paired, so one launch runs both layouts)
    spai = spai_lib

    def build(A, kind, seed):
        dA = upload(spai, A)
        if kind == "fsai":
            M, _ = fsai_precond(spai, A, dA)
            return dA, M, spai.PREC_F64
        if kind == "gnn3d":
            v = W.diffusion3d_node_features(kind_k[0])
            P = spai.build_pattern(dA, spai.PATTERN_FULL)
            mixed = case == "gnn_sell_mixed"
            M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"),
                                 torch.tensor(W.gnn_random_weights(4, 4), device="cuda"), d_node=4,
                                 g_dtype=spai.F32 if mixed else spai.F64, eps=0.3)
            M._keep = P
            return dA, M, spai.PREC_MIXED if mixed else spai.PREC_F64
        P = spai.build_pattern(dA, spai.PATTERN_FULL)
        M = spai.gnn_precond(dA, P, torch.tensor(W.row_average_feature(A), device="cuda"),
                             torch.tensor(W.gnn_random_weights(1, 4), device="cuda"), d_node=1, g_dtype=spai.F32,
                             eps=0.3)
        M._keep = P
        return dA, M, spai.PREC_MIXED

    kind_k = [None]
    if case in ("gnn_sell_mixed", "gnn_csr_f64"):
        A, kind_k[0] = W.diffusion3d(16)
        specs = [(A, "gnn3d", dict(sell=1) if case == "gnn_sell_mixed" else dict(sell=0, staged=1))]
    elif case == "fsai_upper":
        specs = [(W.poisson2d(48), "fsai", dict(sell=0, staged=1))]
    elif case == "graph_direct":
        specs = [(W.graph_laplacian(3000, 24000, seed=5), "graph", dict(sell=0, staged=0))]
    elif case == "graph_sell":
        specs = [(W.graph_laplacian(5000, 40000, seed=9), "graph", dict(sell=1))]
    else:
        specs = [(W.graph_laplacian(2000, 16000, seed=6), "graph", dict(sell=0, staged=1)),
                 (W.aniso2d(60, 30.0, 0.3), "graph", dict(sell=1)),
                 (W.graph_laplacian(500, 4000, seed=7), "graph", dict(sell=0, staged=0)),
                 (W.graph_laplacian(4000, 32000, seed=8), "graph", dict(sell=1))]
    runs = {}
    for on in (0, 1):
        systems, preconds, bs, xs, hs, prec = [], [], [], [], [], None
        for i, (A, kind, sched) in enumerate(specs):
            dA, M, prec = build(A, kind, i)
            S = spai.system_create(dA)
            S.set_schedule(**{flag: on if (flag == "fuse" or len(specs) == 1 or i % 2 == 0) else 0}, **sched)
            assert S.schedule()[flag] == (on if (flag == "fuse" or len(specs) == 1 or i % 2 == 0) else 0)
            systems.append(S), preconds.append(M)
            bs.append(torch.tensor(W.rhs_uniform(A.n, 70 + i), device="cuda"))
            xs.append(torch.zeros(A.n, dtype=torch.float64, device="cuda"))
        if len(specs) == 1:
            h = torch.zeros(100000, dtype=torch.float64, device="cuda")
            r = [spai.system_solve(systems[0], preconds[0], bs[0], xs[0], history=h, precision=prec)]
            hs = [h[:r[0]["history_written"]].clone()]
        else:
            r = spai.pcg_solve_batched(systems, preconds, bs, xs, precision=prec)
        runs[on] = (r, [x.clone() for x in xs], hs)
    (r0, x0, h0), (r1, x1, h1) = runs[0], runs[1]
    for a, b in zip(r0, r1):
        assert a["status"] == 0 and b["status"] == 0
        assert a["iters"] == b["iters"] and a["outer_iters"] == b["outer_iters"]
        assert a["true_rel_res"] <= 1e-8
    for a, b in zip(x0, x1):
        assert torch.equal(a, b)
    for a, b in zip(h0, h1):
        assert torch.equal(a, b)


@pytest.mark.parametrize("mixed", [False, True])
def test_block_layout_matches_oracle(spai_lib, mixed):
    # a matrix made of dense 3 x 3 blocks (Sec. 3.2.2, b = 3) read in the
    # block layout: one column index per block, a lane per block row.
    # float64 with G = D^-1/2 on A's pattern: every ||r_k|| as the oracle's;
    # mixed with the block GNN's G: the float64 rtol, about the float64
    # iteration count, and the scalar layout's iteration count
    spai = spai_lib
    A, feat = W.elastic3d(7)
    dA = upload(spai, A)
    S = spai.system_create(dA)
    lay = S.layout()
    assert lay["block_slices"] == (A.n // 3 + 31) // 32 and lay["block_total"] * 9 >= A.nnz
    b = W.rhs_uniform(A.n, 61)
    pat = spai.build_pattern(dA, spai.PATTERN_FULL)
    if not mixed:
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        diag = A.val[A.colidx == rows]
        g = np.where(A.colidx == rows, 1.0 / np.sqrt(diag[rows]), 0.0)
        M = spai.precond_from_values(pat, torch.tensor(g, device="cuda"), spai.F64, eps=0.0)
        ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g, 0.0), rtol=1e-9)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        h = torch.zeros(20000, dtype=torch.float64, device="cuda")
        r = spai.system_solve(S, M, torch.tensor(b, device="cuda"), x, history=h, rtol=1e-9)
        assert S.schedule()["block"] == 1
        assert r["status"] == 0 and r["iters"] == ref.iters
        k = r["history_written"]
        assert_history_parity(h[:k].cpu().numpy(), ref.history, np.linalg.norm(b))
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        return
    blob = W.gnn_random_weights(feat.shape[1], 4, b=3)
    M = spai.gnn_precond(dA, pat, torch.tensor(feat.astype(np.float32), device="cuda"),
                         torch.tensor(blob, device="cuda"), d_node=feat.shape[1], g_dtype=spai.F32, eps=0.3, block=3)
    its = {}
    for blk in (1, 0):
        S.set_schedule(block=blk)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = spai.system_solve(S, M, torch.tensor(b, device="cuda"), x, precision=spai.PREC_MIXED)
        assert r["status"] == 0
        assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.cpu().numpy(), b) <= 1e-8
        its[blk] = r["iters"]
    assert abs(its[1] - its[0]) <= 0.05 * its[0] + 2, its


def test_block_layout_alone_equals_batch(spai_lib):
    # the block member of a batch (run by the full kernel with a SELL-32 and
    # a CSR member) gives bit-identical results to its solve alone
    spai = spai_lib
    A, feat = W.elastic3d(6)
    dA = upload(spai, A)
    S = spai.system_create(dA)
    pat = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, pat, torch.tensor(feat.astype(np.float32), device="cuda"),
                         torch.tensor(W.gnn_random_weights(feat.shape[1], 4, b=3), device="cuda"),
                         d_node=feat.shape[1], g_dtype=spai.F32, eps=0.3, block=3)
    b = torch.tensor(W.rhs_uniform(A.n, 62), device="cuda")
    x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r1 = spai.system_solve(S, M, b, x1, precision=spai.PREC_MIXED)
    B = W.aniso2d(50, 10.0, 0.4)
    dB = upload(spai, B)
    SB = spai.system_create(dB)
    pB = spai.build_pattern(dB, spai.PATTERN_FULL)
    MB = spai.gnn_precond(dB, pB, torch.tensor(W.row_average_feature(B), device="cuda"),
                          torch.tensor(W.gnn_random_weights(1, 4), device="cuda"), d_node=1, g_dtype=spai.F32, eps=0.3)
    C = W.graph_laplacian(800, 6400, seed=3)
    dC = upload(spai, C)
    SC = spai.system_create(dC)
    SC.set_schedule(sell=0)
    pC = spai.build_pattern(dC, spai.PATTERN_FULL)
    MC = spai.gnn_precond(dC, pC, torch.tensor(W.row_average_feature(C), device="cuda"),
                          torch.tensor(W.gnn_random_weights(1, 4), device="cuda"), d_node=1, g_dtype=spai.F32, eps=0.3)
    bs = [b, torch.tensor(W.rhs_uniform(B.n, 63), device="cuda"), torch.tensor(W.rhs_uniform(C.n, 64), device="cuda")]
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda"), torch.zeros(B.n, dtype=torch.float64, device="cuda"),
          torch.zeros(C.n, dtype=torch.float64, device="cuda")]
    res = spai.pcg_solve_batched([S, SB, SC], [M, MB, MC], bs, xs, precision=spai.PREC_MIXED)
    assert all(r["status"] == 0 for r in res)
    assert res[0]["iters"] == r1["iters"] and torch.equal(xs[0], x1)


@pytest.mark.parametrize("side", [12, 16])
def test_trained_gnn_every_iteration_matches_oracle(spai_lib, side):
    # with the trained weights the float64 iteration is not chaotic (unlike a
    # random-weight G): every ||r_k|| agrees with the oracle's Algorithm 1 at
    # the 1e-10 bar, the iteration counts are equal and x agrees to 1e-8
    import json
    import os
    spai = spai_lib
    wbase = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2510_27517_gb300",
                         "weights", "gnn_diffusion3d_l4")
    blob = np.load(wbase + ".npy").astype(np.float32)
    meta = json.load(open(wbase + ".json"))
    A, k = W.diffusion3d(side, seed=W.BASE_SEED + 77)
    v = W.diffusion3d_node_features(k)
    if meta.get("features") == "logk":
        v = np.ascontiguousarray(v[:, 3:4])
    dA = upload(spai, A)
    P = spai.build_pattern(dA, spai.PATTERN_FULL)
    M = spai.gnn_precond(dA, P, torch.tensor(v, device="cuda"), torch.tensor(blob, device="cuda"),
                         d_node=v.shape[1], g_dtype=spai.F64, eps=1e-4)
    g, _ = M.export(spai.F64)
    b = W.rhs_uniform(A.n, 81)
    ref = pcg.pcg(A.n, A.rowptr, A.colidx, A.val, b, pcg.spai_apply(A.n, A.rowptr, A.colidx, g.cpu().numpy(), 1e-4),
                  rtol=1e-8)
    res, x, hist = gpu_solve(spai, dA, M, b, hist_len=4096)
    assert res["status"] == 0 and ref.status == pcg.CONVERGED
    assert res["iters"] == ref.iters and ref.iters < 200
    k_ = res["history_written"]
    assert k_ == len(ref.history)
    assert_history_parity(hist[:k_], ref.history, np.linalg.norm(b))
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
