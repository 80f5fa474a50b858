"""Continuous-batching server (spai_server_*): requests of different sizes
run together, each result equals the same solve done alone, admission
respects the device-memory cap, and error paths report instead of faulting."""
import time

import numpy as np
import pytest
import torch

import workloads as W
from oracle import fsai, pcg

pytestmark = pytest.mark.gpu


def make_pool(spai, gdt, mats):
    pool = []
    for A in mats:
        dA = spai.CSRMatrix.from_numpy(A.n, A.rowptr, A.colidx, A.val)
        _, _, gv = fsai.fsai_g(A.n, A.rowptr, A.colidx, A.val)
        pat = spai.build_pattern(dA, spai.PATTERN_UPPER)
        M = spai.precond_from_values(pat, torch.tensor(gv, device="cuda"), gdt, eps=0.0)
        S = spai.system_create(dA)
        pool.append((A, dA, S, M))
    return pool


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_results_same_alone_and_in_mix(spai_lib, precision):
    spai = spai_lib
    prec = spai.PREC_MIXED if precision == "mixed" else spai.PREC_F64
    gdt = spai.F32 if precision == "mixed" else spai.F64
    mats = [W.poisson2d(30), W.aniso2d(57, 40.0, 0.3), W.poisson2d(80), W.aniso2d(25, 900.0, 2.5)]
    pool = make_pool(spai, gdt, mats)
    srv = spai.Server(hbm_cap_bytes=1 << 30, max_slots=16, chunk_iters=8, precision=prec)
    ids = [srv.register(S, M) for (_, _, S, M) in pool]
    reqs = []
    for k in range(10):
        i = k % len(pool)
        A = pool[i][0]
        b = torch.tensor(W.rhs_uniform(A.n, 1000 + k)).contiguous()
        x = torch.zeros(A.n, dtype=torch.float64)
        reqs.append((i, b, x, srv.submit(ids[i], b, x)))
    comps = {t: srv.wait(t, 60000) for (_, _, _, t) in reqs}
    srv.close()
    for i, b, x, t in reqs:
        c = comps[t]
        A, dA, S, M = pool[i]
        assert c["status"] == 0 and c["true_rel_res"] <= 1e-8
        assert c["t_submit_us"] <= c["t_admit_us"] <= c["t_done_us"]
        # the same solve alone
        xa = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        ra = spai.system_solve(S, M, b.cuda(), xa, precision=prec)
        assert ra["iters"] == c["iters"]
        xa = xa.cpu().numpy()
        assert np.linalg.norm(x.numpy() - xa) <= 1e-12 * np.linalg.norm(xa)
        assert pcg.true_rel_residual(A.n, A.rowptr, A.colidx, A.val, x.numpy(), b.numpy()) <= 1e-8


def test_admission_under_tight_cap(spai_lib):
    spai = spai_lib
    mats = [W.poisson2d(40), W.poisson2d(40)]
    pool = make_pool(spai, spai.F64, mats)
    n = mats[0].n
    one = 2 * n * 8 + (((n * 8 + 255) // 256) * 256) * 7 + 256   # device bytes of one request
    srv = spai.Server(hbm_cap_bytes=one + 100, max_slots=8, chunk_iters=4)
    ids = [srv.register(S, M) for (_, _, S, M) in pool]
    out = []
    for k in range(4):
        b = torch.tensor(W.rhs_uniform(n, k)).contiguous()
        x = torch.zeros(n, dtype=torch.float64)
        out.append((b, x, srv.submit(ids[k % 2], b, x)))
    comps = sorted((srv.wait(t, 60000) for _, _, t in out), key=lambda c: c["t_admit_us"])
    srv.close()
    # only one request fits: each is admitted after the previous one finished
    for a, b_ in zip(comps, comps[1:]):
        assert b_["t_admit_us"] >= a["t_done_us"]
    assert all(c["status"] == 0 for c in comps)


def test_server_errors(spai_lib):
    spai = spai_lib
    pool = make_pool(spai, spai.F64, [W.poisson2d(20)])
    A, dA, S, M = pool[0]
    srv = spai.Server(hbm_cap_bytes=1000, max_slots=4)
    sid = srv.register(S, M)
    b = torch.ones(A.n, dtype=torch.float64)
    x = torch.zeros(A.n, dtype=torch.float64)
    with pytest.raises(spai.SpaiError) as ei:
        srv.submit(sid, b, x)
    assert ei.value.code == spai.spai.ERR_TOO_LARGE
    with pytest.raises(spai.SpaiError) as ei:
        srv.submit(sid + 5, b, x)
    assert ei.value.code == spai.spai.ERR_NOT_FOUND
    with pytest.raises(spai.SpaiError) as ei:
        srv.wait(12345, 10)
    assert ei.value.code == spai.spai.ERR_NOT_FOUND
    srv.close()


def test_nan_rhs_reports_breakdown(spai_lib):
    spai = spai_lib
    pool = make_pool(spai, spai.F64, [W.poisson2d(20)])
    A, dA, S, M = pool[0]
    srv = spai.Server(hbm_cap_bytes=1 << 28, max_slots=4)
    sid = srv.register(S, M)
    b = torch.tensor(W.rhs_uniform(A.n, 1)).contiguous()
    b[7] = float("nan")
    x = torch.zeros(A.n, dtype=torch.float64)
    t = srv.submit(sid, b, x)
    c = srv.wait(t, 60000)
    b2 = torch.tensor(W.rhs_uniform(A.n, 2)).contiguous()
    x2 = torch.zeros(A.n, dtype=torch.float64)
    c2 = srv.wait(srv.submit(sid, b2, x2), 60000)
    srv.close()
    assert c["status"] != 0          # non-finite scalars end the solve with an error status
    assert c2["status"] == 0         # the server keeps serving
