"""Thin Python binding of the C ABI in include/spai.h (argument marshalling only).

Every computation runs in libspai.so's CUDA kernels; this module only turns
torch tensors into device pointers and C structs into Python objects.  If the
library is missing it raises instead of computing anything on the CPU.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libspai.so")

# status codes (include/spai.h)
OK, ERR_INVALID, ERR_BAD_CSR, ERR_SHAPE, ERR_CUDA, ERR_OOM = 0, -1, -2, -3, -4, -5
ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_TOO_LARGE, ERR_NOT_FOUND = -6, -7, -8, -9, -10
F64, F32, BF16, F16 = 0, 1, 2, 3
PATTERN_FULL, PATTERN_LOWER, PATTERN_UPPER = 0, 1, 2
PREC_F64, PREC_MIXED = 0, 1
CRIT_RESIDUAL, CRIT_PRECOND = 0, 1
MSG_LATENT, MSG_RAW = 0, 1

_TORCH_DT = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}


class SpaiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spai error {code}: {msg}")
        self.code = code


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("val", C.c_void_p), ("dtype", C.c_int32)]


class _GNNW(C.Structure):
    _fields_ = [("blob", C.c_void_p), ("count", C.c_int64), ("d_node", C.c_int32), ("n_layers", C.c_int32),
                ("msg_edge", C.c_int32), ("block", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int64), ("replace_period", C.c_int32),
                ("criterion", C.c_int32), ("precision", C.c_int32), ("inner_rtol", C.c_double),
                ("max_outer", C.c_int32), ("record_history", C.c_int32), ("history", C.c_void_p),
                ("history_len", C.c_int64), ("lanczos", C.c_void_p), ("lanczos_len", C.c_int64)]


class _Res(C.Structure):
    _fields_ = [("iters", C.c_int64), ("outer_iters", C.c_int32), ("status", C.c_int32),
                ("true_rel_res", C.c_double), ("rec_rel_res", C.c_double), ("history_written", C.c_int64),
                ("engine_ms", C.c_double), ("slots", C.c_int64), ("launches", C.c_int32), ("pad", C.c_int32),
                ("lanczos_written", C.c_int64)]


class _Sched(C.Structure):
    _fields_ = [("tile_nnz", C.c_int32), ("items_log2", C.c_int32), ("staged", C.c_int32), ("sell", C.c_int32),
                ("fuse", C.c_int32), ("block", C.c_int32), ("pair", C.c_int32),
                ("tuned", C.c_int32)]


class _AdamW(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("weight_decay", C.c_double), ("max_grad_norm", C.c_double)]


class _Layout(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("max_row", C.c_int32), ("sell_slices", C.c_int32),
                ("sell_total", C.c_int64), ("sell_sorted", C.c_int32), ("block_slices", C.c_int32),
                ("block_total", C.c_int64)]


class _ServeCfg(C.Structure):
    _fields_ = [("hbm_cap_bytes", C.c_int64), ("max_slots", C.c_int32), ("chunk_iters", C.c_int32),
                ("opts", _Opts)]


class _Completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int32), ("iters", C.c_int64), ("outer_iters", C.c_int32),
                ("true_rel_res", C.c_double), ("t_submit_us", C.c_double), ("t_admit_us", C.c_double),
                ("t_done_us", C.c_double)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "spai_last_error": (C.c_char_p, []),
    "spai_version": (C.c_char_p, []),
    "spai_kernel_launches": (C.c_uint64, []),
    "spai_pcg_opts_default": (None, [C.POINTER(_Opts)]),
    "spai_ritz_extremes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    "spai_ritz_kaporin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double)]),
    "spai_sai_loss": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "spai_sai_loss_grad": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "spai_selftest_wait_timeout": (C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.c_void_p]),
    "spai_build_pattern": (C.c_int, [C.POINTER(_CSR), C.c_int32, C.POINTER(C.c_void_p), C.c_void_p]),
    "spai_pattern_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "spai_pattern_export": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.c_void_p]),
    "spai_pattern_destroy": (None, [C.c_void_p]),
    "spai_gnn_grad": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.POINTER(_GNNW), C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "spai_gnn_precond": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.POINTER(_GNNW), C.c_int32,
                                   C.c_double, C.POINTER(C.c_void_p), C.c_void_p]),
    "spai_adamw_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.POINTER(_AdamW), C.c_int64, C.POINTER(C.c_double), C.c_void_p]),
    "spai_precond_from_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                                           C.POINTER(C.c_void_p), C.c_void_p]),
    "spai_precond_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "spai_precond_matrix_norm": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "spai_precond_destroy": (None, [C.c_void_p]),
    "spai_system_create": (C.c_int, [C.POINTER(_CSR), C.c_int32, C.POINTER(C.c_void_p), C.c_void_p]),
    "spai_system_schedule": (C.c_int, [C.c_void_p, C.POINTER(_Sched)]),
    "spai_system_set_schedule": (C.c_int, [C.c_void_p, C.POINTER(_Sched)]),
    "spai_system_info": (C.c_int, [C.c_void_p, C.POINTER(_Layout)]),
    "spai_system_destroy": (None, [C.c_void_p]),
    "spai_pcg_solve": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Opts),
                                 C.POINTER(_Res), C.c_void_p]),
    "spai_system_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Opts),
                                    C.POINTER(_Res), C.c_void_p]),
    "spai_pcg_solve_batched": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(_Opts),
                                         C.POINTER(_Res), C.c_void_p]),
    "spai_pcg_solve_host": (C.c_int, [C.POINTER(_CSR), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Opts),
                                      C.POINTER(_Res), C.c_void_p]),
    "spai_pcg_solve_noalloc": (C.c_int, [C.POINTER(_CSR), C.POINTER(_CSR), C.POINTER(_CSR), C.c_double, C.c_void_p,
                                         C.c_void_p, C.POINTER(_Opts), C.POINTER(_Res), C.c_void_p]),
    "spai_server_create": (C.c_int, [C.POINTER(_ServeCfg), C.POINTER(C.c_void_p)]),
    "spai_server_register": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "spai_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64)]),
    "spai_server_poll": (C.c_int, [C.c_void_p, C.POINTER(_Completion), C.c_int32, C.POINTER(C.c_int32)]),
    "spai_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(_Completion)]),
    "spai_server_destroy": (C.c_int, [C.c_void_p]),
}


def exported_symbols():
    """Names the header declares (the binding's view of the ABI)."""
    return list(_SIGS)


def lib():
    """Load libspai.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libspai.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (rt, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = rt
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise SpaiError(rc, lib().spai_last_error().decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _check_vec(t, n, name, cuda=True):
    """A contiguous float64 vector of at least n entries on the expected side
    (the library reads and writes n entries through its raw pointer)."""
    assert t.dtype == torch.float64, f"{name} must be float64"
    assert t.is_cuda == cuda, f"{name} must be a {'device' if cuda else 'host'} tensor"
    assert t.is_contiguous(), f"{name} must be contiguous"
    assert t.numel() >= n, f"{name} has {t.numel()} entries, the system has {n} rows"


# ---------------------------------------------------------------------------
@dataclasses.dataclass
class CSRMatrix:
    """Device CSR of float64 A (int32 indices)."""
    n: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    val: torch.Tensor

    @staticmethod
    def from_numpy(n, rowptr, colidx, val, device="cuda"):
        return CSRMatrix(int(n), torch.as_tensor(rowptr, dtype=torch.int32).to(device),
                         torch.as_tensor(colidx, dtype=torch.int32).to(device),
                         torch.as_tensor(val, dtype=torch.float64).to(device))

    @property
    def nnz(self):
        return int(self.colidx.numel())

    def _c(self):
        self._keep = _CSR(self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(),
                          self.val.data_ptr(), F64)
        return self._keep


class _Handle:
    _destroy = None

    def __init__(self, h):
        self.h = h

    def close(self):
        if self.h:
            getattr(lib(), self._destroy)(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pattern(_Handle):
    _destroy = "spai_pattern_destroy"

    def info(self):
        n, m = C.c_int64(), C.c_int64()
        _check(lib().spai_pattern_info(self.h, C.byref(n), C.byref(m)))
        return n.value, m.value

    def export(self):
        n, m = self.info()
        dev = torch.device("cuda")
        out = [torch.empty(n + 1, dtype=torch.int32, device=dev), torch.empty(m, dtype=torch.int32, device=dev),
               torch.empty(n + 1, dtype=torch.int32, device=dev), torch.empty(m, dtype=torch.int32, device=dev),
               torch.empty(m, dtype=torch.int32, device=dev)]
        _check(lib().spai_pattern_export(self.h, *[_ptr(t) for t in out], _stream()))
        return dict(zip(["rowptr", "colidx", "t_rowptr", "t_colidx", "perm"], out))


class Precond(_Handle):
    _destroy = "spai_precond_destroy"

    def __init__(self, h, pattern):
        super().__init__(h)
        self.pattern = pattern

    def export(self, dtype=F64):
        _, m = self.pattern.info()
        g = torch.empty(m, dtype=_TORCH_DT[dtype], device="cuda")
        gt = torch.empty(m, dtype=_TORCH_DT[dtype], device="cuda")
        _check(lib().spai_precond_export(self.h, _ptr(g), _ptr(gt), dtype, _stream()))
        return g, gt

    def matrix_norm(self):
        v = C.c_double()
        _check(lib().spai_precond_matrix_norm(self.h, C.byref(v)))
        return v.value


class System(_Handle):
    _destroy = "spai_system_destroy"

    def __init__(self, h, A):
        super().__init__(h)
        self.A = A

    def schedule(self):
        sc = _Sched()
        _check(lib().spai_system_schedule(self.h, C.byref(sc)))
        return {k: getattr(sc, k) for k, _ in _Sched._fields_}

    def layout(self):
        lo = _Layout()
        _check(lib().spai_system_info(self.h, C.byref(lo)))
        return {k: getattr(lo, k) for k, _ in _Layout._fields_}

    def set_schedule(self, tile_nnz=0, items_log2=0, staged=1, sell=1, fuse=1, block=1, pair=None):
        """pair=None: paired vectors where the rows were sorted by length (the default at creation)."""
        if pair is None:
            pair = 1 if self.layout()["sell_sorted"] else 0
        sc = _Sched(tile_nnz, items_log2, staged, sell, fuse, block, pair, 0)
        _check(lib().spai_system_set_schedule(self.h, C.byref(sc)))


def build_pattern(A: CSRMatrix, kind=PATTERN_FULL, stream=None) -> Pattern:
    h = C.c_void_p()
    _check(lib().spai_build_pattern(C.byref(A._c()), kind, C.byref(h), _stream(stream)))
    return Pattern(h.value)


def gnn_precond(A: CSRMatrix, P: Pattern, node_feat: torch.Tensor, blob: torch.Tensor, d_node: int,
                n_layers: int = 4, msg_edge=MSG_LATENT, g_dtype=F32, eps=1e-4, block=1, stream=None) -> Precond:
    """block=3: A made of dense 3 x 3 blocks, node_feat one row per block row."""
    assert node_feat.dtype == torch.float32 and node_feat.is_contiguous()
    assert blob.dtype == torch.float32 and blob.is_contiguous()
    assert node_feat.numel() == (A.n // max(1, block)) * d_node, "node_feat must hold (n / block) x d_node values"
    w = _GNNW(blob.data_ptr(), blob.numel(), d_node, n_layers, msg_edge, block)
    h = C.c_void_p()
    _check(lib().spai_gnn_precond(C.byref(A._c()), P.h, _ptr(node_feat), C.byref(w), g_dtype, float(eps),
                                  C.byref(h), _stream(stream)))
    return Precond(h.value, P)


def gnn_grad(A: CSRMatrix, P: Pattern, node_feat: torch.Tensor, blob: torch.Tensor, dG: torch.Tensor, d_node: int,
             n_layers: int = 4, msg_edge=MSG_LATENT, block=1, stream=None) -> torch.Tensor:
    """Gradient of sum(dG * G) with respect to the weight blob (float64);
    block=3 as in gnn_precond."""
    assert node_feat.dtype == torch.float32 and node_feat.is_contiguous()
    assert blob.dtype == torch.float32 and blob.is_contiguous()
    assert dG.dtype == torch.float64 and dG.is_contiguous() and dG.is_cuda
    nodes = A.n // max(1, block)
    assert node_feat.numel() == nodes * d_node, "node_feat must hold (n / block) x d_node values"
    assert dG.numel() == P.info()[1], "dG must hold one value per entry of G"
    w = _GNNW(blob.data_ptr(), blob.numel(), d_node, n_layers, msg_edge, block)
    out = torch.empty(blob.numel(), dtype=torch.float64, device=blob.device)
    _check(lib().spai_gnn_grad(C.byref(A._c()), P.h, _ptr(node_feat), C.byref(w), _ptr(dG), _ptr(out),
                               _stream(stream)))
    return out


def adamw_step(master: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, blob: torch.Tensor,
               step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01, max_grad_norm=0.0,
               stream=None) -> float:
    """One AdamW step (spai_adamw_step) on the float64 master weights, moments
    m and v, writing the float32 blob; returns the gradient's 2-norm."""
    count = master.numel()
    for t in (master, m, v, grad):
        _check_vec(t, count, "AdamW state")
    assert blob.dtype == torch.float32 and blob.is_cuda and blob.is_contiguous() and blob.numel() == count
    cfg = _AdamW(lr, beta1, beta2, eps, weight_decay, max_grad_norm)
    gn = C.c_double()
    _check(lib().spai_adamw_step(_ptr(master), _ptr(m), _ptr(v), _ptr(grad), _ptr(blob), count, C.byref(cfg), step,
                                 C.byref(gn), _stream(stream)))
    return gn.value


def precond_from_values(P: Pattern, g_val: torch.Tensor, g_dtype=F64, eps=0.0, stream=None) -> Precond:
    vdt = {torch.float64: F64, torch.float32: F32}[g_val.dtype]
    h = C.c_void_p()
    _check(lib().spai_precond_from_values(P.h, _ptr(g_val.contiguous()), vdt, g_dtype, float(eps), C.byref(h),
                                          _stream(stream)))
    return Precond(h.value, P)


def system_create(A: CSRMatrix, autotune=False, stream=None) -> System:
    h = C.c_void_p()
    _check(lib().spai_system_create(C.byref(A._c()), 1 if autotune else 0, C.byref(h), _stream(stream)))
    return System(h.value, A)


def make_opts(rtol=1e-8, max_iter=0, replace_period=50, criterion=CRIT_RESIDUAL, precision=PREC_F64,
              inner_rtol=0.1, max_outer=0, history: torch.Tensor | None = None,
              lanczos: torch.Tensor | None = None) -> _Opts:
    o = _Opts()
    lib().spai_pcg_opts_default(C.byref(o))
    o.rtol, o.max_iter, o.replace_period, o.criterion = rtol, max_iter, replace_period, criterion
    o.precision, o.inner_rtol, o.max_outer = precision, inner_rtol, max_outer
    if history is not None:
        assert history.dtype == torch.float64 and history.is_cuda
        o.record_history, o.history, o.history_len = 1, history.data_ptr(), history.numel()
    if lanczos is not None:
        assert lanczos.dtype == torch.float64 and lanczos.is_cuda and lanczos.numel() % 2 == 0
        o.lanczos, o.lanczos_len = lanczos.data_ptr(), lanczos.numel() // 2
    return o


def _host_f64(a):
    t = torch.as_tensor(a, dtype=torch.float64).cpu().contiguous()
    return t, C.c_void_p(t.data_ptr())


def sai_loss(A: CSRMatrix, M: Precond, w: torch.Tensor, stream=None) -> torch.Tensor:
    """SAI loss of every probe column of w (n x k float64 on the device, k <= 32)."""
    assert w.dtype == torch.float64 and w.is_cuda and w.dim() == 2 and w.shape[0] == A.n
    w = w.contiguous()
    out = torch.empty(w.shape[1], dtype=torch.float64, device=w.device)
    _check(lib().spai_sai_loss(C.byref(A._c()), M.h, _ptr(w), w.shape[1], _ptr(out), _stream(stream)))
    return out


def sai_loss_grad(A: CSRMatrix, M: Precond, w: torch.Tensor, stream=None):
    """Per-probe SAI loss and the gradient of its mean with respect to G's
    stored values (float64, G's CSR order)."""
    assert w.dtype == torch.float64 and w.is_cuda and w.dim() == 2 and w.shape[0] == A.n
    w = w.contiguous()
    loss = torch.empty(w.shape[1], dtype=torch.float64, device=w.device)
    grad = torch.empty(M.pattern.info()[1], dtype=torch.float64, device=w.device)
    _check(lib().spai_sai_loss_grad(C.byref(A._c()), M.h, _ptr(w), w.shape[1], _ptr(loss), _ptr(grad),
                                    _stream(stream)))
    return loss, grad


def selftest_wait_timeout(limit_us=20000, stream=None) -> bool:
    """True when the device-side bounded waits gave up and reported it."""
    d = C.c_int32()
    _check(lib().spai_selftest_wait_timeout(limit_us, C.byref(d), _stream(stream)))
    return bool(d.value)


def ritz_extremes(alpha, beta):
    """(lam_min, lam_max) of the Lanczos matrix of k PCG steps (spai_ritz_extremes)."""
    ta, pa = _host_f64(alpha)
    tb, pb = _host_f64(beta)
    lo, hi = C.c_double(), C.c_double()
    _check(lib().spai_ritz_extremes(pa, pb, ta.numel(), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def ritz_kaporin(alpha, beta):
    """Kaporin's condition number by Gauss quadrature on the Lanczos matrix."""
    ta, pa = _host_f64(alpha)
    tb, pb = _host_f64(beta)
    v = C.c_double()
    _check(lib().spai_ritz_kaporin(pa, pb, ta.numel(), C.byref(v)))
    return v.value


def _res_dict(r: _Res):
    return {"iters": r.iters, "outer_iters": r.outer_iters, "status": r.status, "true_rel_res": r.true_rel_res,
            "rec_rel_res": r.rec_rel_res, "history_written": r.history_written, "engine_ms": r.engine_ms,
            "slots": r.slots, "launches": r.launches, "lanczos_written": r.lanczos_written}


def kernel_launches() -> int:
    """CUDA kernels launched by the library so far in this process."""
    return int(lib().spai_kernel_launches())


def _solve_rc(rc):
    if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        _check(rc)


def pcg_solve(A: CSRMatrix, M: Precond, b: torch.Tensor, x: torch.Tensor, stream=None, **kw):
    _check_vec(b, A.n, "b")
    _check_vec(x, A.n, "x")
    o = make_opts(**kw)
    r = _Res()
    _solve_rc(lib().spai_pcg_solve(C.byref(A._c()), M.h, _ptr(b), _ptr(x), C.byref(o), C.byref(r), _stream(stream)))
    return _res_dict(r)


def system_solve(S: System, M: Precond, b: torch.Tensor, x: torch.Tensor, stream=None, **kw):
    _check_vec(b, S.A.n, "b")
    _check_vec(x, S.A.n, "x")
    o = make_opts(**kw)
    r = _Res()
    _solve_rc(lib().spai_system_solve(S.h, M.h, _ptr(b), _ptr(x), C.byref(o), C.byref(r), _stream(stream)))
    return _res_dict(r)


def pcg_solve_batched(systems, preconds, bs, xs, stream=None, **kw):
    n = len(systems)
    assert len(preconds) == n and len(bs) == n and len(xs) == n
    for S, b, x in zip(systems, bs, xs):
        _check_vec(b, S.A.n, "b")
        _check_vec(x, S.A.n, "x")
    arr = lambda vals: (C.c_void_p * n)(*vals)  # noqa: E731
    o = make_opts(**kw)
    res = (_Res * n)()
    _solve_rc(lib().spai_pcg_solve_batched(n, arr([s.h for s in systems]), arr([m.h for m in preconds]),
                                           arr([b.data_ptr() for b in bs]), arr([x.data_ptr() for x in xs]),
                                           C.byref(o), res, _stream(stream)))
    return [_res_dict(r) for r in res]


def pcg_solve_host(A: CSRMatrix, M: Precond, b_host, x_host, stream=None, **kw):
    """b_host, x_host: contiguous float64 CPU tensors (pinned for speed)."""
    _check_vec(b_host, A.n, "b_host", cuda=False)
    _check_vec(x_host, A.n, "x_host", cuda=False)
    o = make_opts(**kw)
    r = _Res()
    _solve_rc(lib().spai_pcg_solve_host(C.byref(A._c()), M.h, C.c_void_p(b_host.data_ptr()),
                                        C.c_void_p(x_host.data_ptr()), C.byref(o), C.byref(r), _stream(stream)))
    return _res_dict(r)


def pcg_solve_noalloc(A: CSRMatrix, G: CSRMatrix, GT: CSRMatrix, eps: float, b: torch.Tensor, x: torch.Tensor,
                      stream=None, **kw):
    """float64 PCG that allocates no device memory (spai_pcg_solve_noalloc):
    G and GT are device CSRs of G and its explicit transpose; all working
    memory comes from the library's static device scratch array."""
    _check_vec(b, A.n, "b")
    _check_vec(x, A.n, "x")
    assert G.n == A.n and GT.n == A.n and G.nnz == GT.nnz
    o = make_opts(**kw)
    r = _Res()
    a_c, g_c, gt_c = A._c(), G._c(), GT._c()
    _solve_rc(lib().spai_pcg_solve_noalloc(C.byref(a_c), C.byref(g_c), C.byref(gt_c), float(eps), _ptr(b), _ptr(x),
                                           C.byref(o), C.byref(r), _stream(stream)))
    return _res_dict(r)


class Server(_Handle):
    """Continuous-batching solve server (spai_server_*)."""
    _destroy = "spai_server_destroy"

    def __init__(self, hbm_cap_bytes=120 << 30, max_slots=64, chunk_iters=16, **kw):
        cfg = _ServeCfg()
        cfg.hbm_cap_bytes, cfg.max_slots, cfg.chunk_iters = hbm_cap_bytes, max_slots, chunk_iters
        cfg.opts = make_opts(**kw)
        h = C.c_void_p()
        _check(lib().spai_server_create(C.byref(cfg), C.byref(h)))
        super().__init__(h.value)
        self._refs = []

    def register(self, S: System, M: Precond) -> int:
        sid = C.c_int64()
        _check(lib().spai_server_register(self.h, S.h, M.h, C.byref(sid)))
        self._refs.append((S, M))
        return sid.value

    def submit(self, sys_id: int, b_host: torch.Tensor, x_host: torch.Tensor) -> int:
        t = C.c_uint64()
        self._refs.append((b_host, x_host))
        _check(lib().spai_server_submit(self.h, sys_id, C.c_void_p(b_host.data_ptr()),
                                        C.c_void_p(x_host.data_ptr()), C.byref(t)))
        return t.value

    def poll(self, max_n=256):
        out = (_Completion * max_n)()
        cnt = C.c_int32()
        _check(lib().spai_server_poll(self.h, out, max_n, C.byref(cnt)))
        return [self._comp(out[i]) for i in range(cnt.value)]

    def wait(self, ticket: int, timeout_ms: int = 60000):
        c = _Completion()
        _check(lib().spai_server_wait(self.h, ticket, timeout_ms, C.byref(c)))
        return self._comp(c)

    @staticmethod
    def _comp(c):
        return {"ticket": c.ticket, "status": c.status, "iters": c.iters, "outer_iters": c.outer_iters,
                "true_rel_res": c.true_rel_res, "t_submit_us": c.t_submit_us, "t_admit_us": c.t_admit_us,
                "t_done_us": c.t_done_us}
