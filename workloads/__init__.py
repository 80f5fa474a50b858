"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *makes inputs*: sparse SPD matrices in CSR form, right-hand
sides, node features and random GNN weights.  It holds none of the solver's or
the GNN's arithmetic (no norms of A, no preconditioner, no CG, no MLP), so the
CPU oracle and the CUDA path can both consume what it produces without sharing
any part of the method.

The workloads stand in for the paper's datasets (Sec. 4.1 and App. C): the
TetWild FEM meshes, the hyperelastic beam and the P P^T + eps I matrices are
not available, so grid stencils and random graphs with the same structure
(symmetric pattern, diagonal present, 5-30 nonzeros per row) are generated
here.  Every generator is deterministic in its seed.

CSR convention used everywhere: int32 ``rowptr`` (n+1) and ``colidx`` (nnz),
columns strictly ascending in each row, no duplicates, diagonal present,
float64 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2510_27517


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox 4x64) for a given integer seed."""
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1)))


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz]
    val: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.colidx] = self.val
        return d


def coo_to_csr(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Sort (row, col) pairs and build CSR.  Duplicates are a generator bug."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate (row, col) entries")
    rows = rows[order]
    cols = cols[order]
    vals = np.asarray(vals, dtype=np.float64)[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def dense_to_csr(a: np.ndarray) -> CSR:
    """Pattern = entries that are nonzero or on the diagonal."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    mask = (a != 0) | np.eye(n, dtype=bool)
    r, c = np.nonzero(mask)
    return coo_to_csr(n, r, c, a[r, c])


# ---------------------------------------------------------------------------
# Grid stencils
# ---------------------------------------------------------------------------

def poisson2d(N: int) -> CSR:
    """5-point -Laplacian on an N x N interior grid, Dirichlet rows eliminated.

    Diagonal 4, neighbours -1.  n = N^2, nnz = 5 N^2 - 4 N (20,224 for N=64).
    """
    n = N * N
    idx = np.arange(n).reshape(N, N)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 4.0)]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        i0, i1 = max(0, -di), N - max(0, di)
        j0, j1 = max(0, -dj), N - max(0, dj)
        src = idx[i0:i1, j0:j1]
        dst = idx[i0 + di:i1 + di, j0 + dj:j1 + dj]
        rows.append(src.ravel())
        cols.append(dst.ravel())
        vals.append(np.full(src.size, -1.0))
    return coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def gaussian_random_field(shape, corr_len: float, seed: int) -> np.ndarray:
    """Unit-variance periodic Gaussian random field.

    White N(0,1) noise convolved (via FFT, separably) with a Gaussian kernel of
    standard deviation corr_len / sqrt(2) cells, then renormalised to zero mean
    and unit sample standard deviation (a constant zero field when the grid is
    so much smaller than the correlation length that no variation survives).
    """
    g = rng(seed)
    w = g.standard_normal(shape)
    sd = corr_len / math.sqrt(2.0)
    f = np.fft.fftn(w)
    for ax, m in enumerate(shape):
        k = np.fft.fftfreq(m)  # cycles per cell
        kern = np.exp(-2.0 * (math.pi * k * sd) ** 2)  # FT of the Gaussian kernel
        sh = [1] * len(shape)
        sh[ax] = m
        f = f * kern.reshape(sh)
    field = np.real(np.fft.ifftn(f))
    field -= field.mean()
    sd_f = field.std()
    if not sd_f > 1e-12:   # grid much smaller than the correlation length: a constant field
        return np.zeros(shape)
    field /= sd_f
    return field


def diffusion3d(N: int, sigma: float = 1.5, corr_len: float = 8.0, seed: int = BASE_SEED + 2):
    """Cell-centred finite-volume -div(k grad u) on N^3 cells, 7-point stencil.

    k = exp(sigma * g) with g a unit-variance Gaussian random field of
    correlation length ``corr_len`` cells.  Face transmissibility between cells
    i, j is the harmonic mean 2 k_i k_j / (k_i + k_j); a Dirichlet boundary face
    contributes 2 k_i to the diagonal.  n = N^3, nnz = 7 n - 6 N^2.

    Returns (A, k) with k the cell coefficient array of shape (N, N, N).
    """
    g = gaussian_random_field((N, N, N), corr_len, seed)
    k = np.exp(sigma * g)
    n = N ** 3
    idx = np.arange(n).reshape(N, N, N)
    diag = np.zeros((N, N, N))
    rows, cols, vals = [], [], []
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, N - 1)
        hi[ax] = slice(1, N)
        ki, kj = k[tuple(lo)], k[tuple(hi)]
        t = 2.0 * ki * kj / (ki + kj)
        diag[tuple(lo)] += t
        diag[tuple(hi)] += t
        a, b = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [-t.ravel(), -t.ravel()]
        # Dirichlet faces on both ends of this axis
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = 0
        last[ax] = N - 1
        diag[tuple(first)] += 2.0 * k[tuple(first)]
        diag[tuple(last)] += 2.0 * k[tuple(last)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return A, k


def diffusion3d_node_features(k: np.ndarray) -> np.ndarray:
    """Heat-equation-like node features (App. C): cell position in [-1,1]^3
    and the log of the cell coefficient.  Shape [n, 4], float32."""
    N = k.shape[0]
    c = (np.arange(N) + 0.5) / N * 2.0 - 1.0
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    f = np.stack([X.ravel(), Y.ravel(), Z.ravel(), np.log(k).ravel()], axis=1)
    return f.astype(np.float32)


def aniso2d(N: int, a: float, theta: float) -> CSR:
    """2D anisotropic diffusion -div(K grad u), K = R diag(1, 1/a) R^T.

    5-point part kxx/kyy plus a rotated cross term: the mixed derivative
    -2 kxy u_xy is discretised with central differences, giving corner weights
    -kxy/2 on (+1,+1),(-1,-1) and +kxy/2 on (+1,-1),(-1,+1).  Dirichlet rows
    eliminated, so nnz = (3N-2)^2.  SPD whenever K is SPD.
    """
    c, s = math.cos(theta), math.sin(theta)
    l1, l2 = 1.0, 1.0 / a
    kxx = c * c * l1 + s * s * l2
    kyy = s * s * l1 + c * c * l2
    kxy = c * s * (l1 - l2)
    n = N * N
    idx = np.arange(n).reshape(N, N)
    rows, cols, vals = [], [], []
    stencil = {
        (0, 0): 2 * kxx + 2 * kyy,
        (1, 0): -kxx, (-1, 0): -kxx,
        (0, 1): -kyy, (0, -1): -kyy,
        (1, 1): -kxy / 2, (-1, -1): -kxy / 2,
        (1, -1): kxy / 2, (-1, 1): kxy / 2,
    }
    for (di, dj), w in stencil.items():
        i0, i1 = max(0, -di), N - max(0, di)
        j0, j1 = max(0, -dj), N - max(0, dj)
        src = idx[i0:i1, j0:j1]
        dst = idx[i0 + di:i1 + di, j0 + dj:j1 + dj]
        rows.append(src.ravel())
        cols.append(dst.ravel())
        vals.append(np.full(src.size, w))
    return coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def aniso2d_batch(count: int, seed: int = BASE_SEED + 4, side_lo: int = 32, side_hi: int = 512):
    """Batch of anisotropic systems: side log-uniform in [side_lo, side_hi],
    anisotropy ratio log-uniform in [1, 1e3], angle uniform in [0, pi)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        N = int(round(math.exp(g.uniform(math.log(side_lo), math.log(side_hi)))))
        a = math.exp(g.uniform(0.0, math.log(1e3)))
        th = g.uniform(0.0, math.pi)
        out.append((N, a, th))
    return out


# ---------------------------------------------------------------------------
# Random graph Laplacian
# ---------------------------------------------------------------------------

def graph_laplacian(n: int, m: int, seed: int = BASE_SEED + 3, wlo: float = 1e-3, whi: float = 1.0,
                    shift_rel: float = 1e-4) -> CSR:
    """Weighted Laplacian of a G(n, m) random graph plus a small diagonal shift.

    m distinct undirected non-loop edges, weights log-uniform in [wlo, whi].
    A = L_w + shift_rel * mean(diag L_w) * I.  nnz = n + 2 m.
    """
    g = rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = int((m - keys.size) * 1.05) + 16
        u = g.integers(0, n, size=need, dtype=np.int64)
        v = g.integers(0, n, size=need, dtype=np.int64)
        keep = u != v
        u, v = u[keep], v[keep]
        lo, hi = np.minimum(u, v), np.maximum(u, v)
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    keys = g.permutation(keys)[:m]
    lo, hi = keys // n, keys % n
    w = np.exp(g.uniform(math.log(wlo), math.log(whi), size=m))
    deg = np.bincount(lo, weights=w, minlength=n) + np.bincount(hi, weights=w, minlength=n)
    shift = shift_rel * deg.mean()
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    vals = np.concatenate([-w, -w, deg + shift])
    return coo_to_csr(n, rows, cols, vals)


def row_average_feature(A: CSR) -> np.ndarray:
    """Synthetic-dataset node feature (App. C): the i-th row average of A,
    taken over the row's stored entries.  Shape [n, 1], float32."""
    s = np.add.reduceat(A.val, A.rowptr[:-1].astype(np.int64)) if A.nnz else np.zeros(A.n)
    cnt = np.diff(A.rowptr)
    s = np.where(cnt > 0, s, 0.0)
    return (s / np.maximum(cnt, 1)).reshape(-1, 1).astype(np.float32)


# ---------------------------------------------------------------------------
# Random SPD matrices for small tests
# ---------------------------------------------------------------------------

def random_spd_sparse(n: int, density: float, seed: int, diag_boost: float = 1.0) -> CSR:
    """Symmetric sparse matrix with a random pattern, made SPD by diagonal
    dominance: A_ii = sum_j |A_ij| + diag_boost."""
    g = rng(seed)
    m = max(1, int(density * n * n / 2))
    u = g.integers(0, n, size=m)
    v = g.integers(0, n, size=m)
    keep = u != v
    lo, hi = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    keys = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = keys // n, keys % n
    w = g.uniform(-1.0, 1.0, size=keys.size)
    absrow = np.bincount(lo, weights=np.abs(w), minlength=n) + np.bincount(hi, weights=np.abs(w), minlength=n)
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    vals = np.concatenate([w, w, absrow + diag_boost])
    return coo_to_csr(n, rows, cols, vals)


def elastic3d(N: int, seed: int = BASE_SEED + 8, shift: float = 1e-3):
    """Block-sparse SPD system with 3 x 3 blocks on an N^3 node grid (the
    shape of the paper's hyperelastic systems: 3 unknowns per node, App. C).

    Every grid edge (i, j) with unit direction n_ij and a log-normal weight
    k_ij adds k_ij (e_i - e_j)(e_i - e_j)^T (x) B_ij, B_ij = I + n n^T
    (a spring that is stiffer along the edge), plus shift * mean(diag) on the
    diagonal; SPD.  Returns the scalar CSR of size 3 N^3 with dense 3 x 3
    blocks (each block row's three scalar rows list the same blocks in column
    order, 3 entries per block), and the node features: position in
    [-1, 1]^3 and a boundary flag (d_node = 4, as the paper's input: position
    and a one-hot Dirichlet indicator)."""
    g = rng(seed)
    nn = N ** 3
    idx = np.arange(nn).reshape(N, N, N)
    blocks = {}
    def add(i, j, M):
        key = (int(i), int(j))
        blocks[key] = blocks.get(key, 0) + M
    diag = np.zeros((nn, 3, 3))
    for ax in range(3):
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[ax] = slice(0, N - 1)
        sl_b[ax] = slice(1, N)
        a = idx[tuple(sl_a)].ravel()
        b = idx[tuple(sl_b)].ravel()
        k = np.exp(0.5 * g.standard_normal(a.size))
        B = np.eye(3)
        B[ax, ax] += 1.0
        for ii, jj, kk in zip(a, b, k):
            M = kk * B
            diag[ii] += M
            diag[jj] += M
            add(ii, jj, -M)
            add(jj, ii, -M)
    dmean = np.mean(np.einsum("ikk->ik", diag))
    for i in range(nn):
        add(i, i, diag[i] + shift * dmean * np.eye(3))
    keys = sorted(blocks)
    brow = np.array([k[0] for k in keys])
    bcol = np.array([k[1] for k in keys])
    bval = np.array([blocks[k] for k in keys])          # (nnzb, 3, 3)
    rows, cols, vals = [], [], []
    for r in range(3):
        for c in range(3):
            rows.append(3 * brow + r)
            cols.append(3 * bcol + c)
            vals.append(bval[:, r, c])
    A = coo_to_csr(3 * nn, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    t = np.linspace(-1.0, 1.0, N)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    bnd = ((idx == idx) & ((np.abs(X) == 1) | (np.abs(Y) == 1) | (np.abs(Z) == 1))).astype(np.float64)
    feat = np.stack([X.ravel(), Y.ravel(), Z.ravel(), bnd.ravel()], axis=1).astype(np.float32)
    return A, feat


def ppt_synthetic(n: int, density: float = 3e-4, eps: float = 1e-4, seed: int = BASE_SEED + 6) -> CSR:
    """The paper's synthetic system A = P P^T + eps I (App. C): P is n x n
    with density * n^2 entries at uniformly random distinct positions and
    standard normal values; A has about 4x that density (1.2e-3 for the
    paper's 3e-4) and is SPD for eps > 0."""
    import scipy.sparse as sp
    g = rng(seed)
    m = max(1, int(round(density * n * n)))
    keys = np.unique(g.integers(0, n * n, size=int(m * 1.05) + 8, dtype=np.int64))
    keys = g.permutation(keys)[:m]
    P = sp.csr_matrix((g.standard_normal(keys.size), (keys // n, keys % n)), shape=(n, n))
    A = (P @ P.T + eps * sp.identity(n, format="csr")).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return CSR(n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def ppt_batch(count: int, seed: int = BASE_SEED + 7, n_lo: int = 12_000, n_hi: int = 24_000):
    """Sizes and seeds of a batch of synthetic systems, n uniform in [n_lo, n_hi]."""
    g = rng(seed)
    return [(int(g.integers(n_lo, n_hi + 1)), int(g.integers(0, 2 ** 31))) for _ in range(count)]


def random_dense_spd(n: int, seed: int, cond: float = 10.0) -> np.ndarray:
    """Dense SPD matrix with eigenvalues log-spaced in [1, cond]."""
    g = rng(seed)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.exp(np.linspace(0.0, math.log(cond), n))
    a = (q * lam) @ q.T
    return 0.5 * (a + a.T)


# ---------------------------------------------------------------------------
# Right-hand sides and GNN weights
# ---------------------------------------------------------------------------

def rhs_uniform(n: int, seed: int) -> np.ndarray:
    return rng(seed).uniform(-1.0, 1.0, size=n)


def rhs_normal(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(n)


HIDDEN = 24  # width d of every hidden layer and latent vector (Sec. 4.1)


def gnn_layer_shapes(d_node: int, n_layers: int, msg_raw_edge: bool = False, d_edge: int = 1, b: int = 1):
    """(name, fan_in, fan_out) for every MLP, in blob order:
    E_n, E_e, then (f_m, f_v, f_e) per message-passing layer, then D.
    Each MLP is Linear(fan_in -> 24), ReLU, Linear(24 -> fan_out)."""
    d = HIDDEN
    shapes = [("E_n", d_node, d), ("E_e", d_edge, d)]
    for t in range(n_layers):
        shapes.append((f"f_m{t}", 2 * d + (d_edge if msg_raw_edge else d), d))
        shapes.append((f"f_v{t}", d, d))
        shapes.append((f"f_e{t}", 3 * d, d))
    shapes.append(("D", d, b * b))
    return shapes


def gnn_param_count(d_node: int, n_layers: int, msg_raw_edge: bool = False, b: int = 1) -> int:
    tot = 0
    for _, fi, fo in gnn_layer_shapes(d_node, n_layers, msg_raw_edge, d_edge=b * b, b=b):
        tot += HIDDEN * fi + HIDDEN + fo * HIDDEN + fo
    return tot


def gnn_random_weights(d_node: int, n_layers: int = 4, seed: int = BASE_SEED + 100,
                       msg_raw_edge: bool = False, b: int = 1) -> np.ndarray:
    """Flat float32 weight blob with seeded U(-1/sqrt(fan_in), 1/sqrt(fan_in))
    initialisation of every weight and bias.

    Per MLP the layout is [W1 (24 x fan_in, row-major), b1 (24),
    W2 (fan_out x 24, row-major), b2 (fan_out)]; MLPs in the order of
    gnn_layer_shapes; b x b blocks make the edge input and the decoder
    output b^2 wide.
    """
    g = rng(seed)
    parts = []
    for _, fi, fo in gnn_layer_shapes(d_node, n_layers, msg_raw_edge, d_edge=b * b, b=b):
        a1 = 1.0 / math.sqrt(fi)
        parts.append(g.uniform(-a1, a1, size=HIDDEN * fi))
        parts.append(g.uniform(-a1, a1, size=HIDDEN))
        a2 = 1.0 / math.sqrt(HIDDEN)
        parts.append(g.uniform(-a2, a2, size=fo * HIDDEN))
        parts.append(g.uniform(-a2, a2, size=fo))
    return np.concatenate(parts).astype(np.float32)
