// GNN reverse pass on the GPU (Sec. 3.3: the GNN of Sec. 3.2.2 is trained on
// the SAI loss): the CUDA executor of the driver in gnn_grad.cuh.  One thread
// per element (edge or node) for the MLPs, gathers and row sums; the weight
// gradients are sums over elements, taken in chunks of kChunk elements whose
// partials are added in chunk order (deterministic).  float64 throughout.
#include <cstring>
#include <deque>
#include <vector>

#include "internal.cuh"
#include "gnn_grad.cuh"

namespace spai {
namespace {

using gg::H;
using gg::Mlp;

constexpr int kThreads = 256;

int grid_for(int64_t work) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

#define GG_LOOP(i, N) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (N); \
                           i += (int64_t)gridDim.x * blockDim.x)

__global__ void rows_kernel(const int32_t* __restrict__ rp, int64_t n, int32_t* __restrict__ rows) {
  GG_LOOP(i, n) for (int e = rp[i]; e < rp[i + 1]; ++e) rows[e] = (int32_t)i;
}

__global__ void inv_kernel(const int32_t* __restrict__ perm, int64_t nnz, int32_t* __restrict__ inv) {
  GG_LOOP(e, nnz) inv[perm[e]] = (int32_t)e;
}

__global__ void to_f64_kernel(const float* __restrict__ in, int64_t count, double* __restrict__ out) {
  GG_LOOP(k, count) out[k] = (double)in[k];
}

__global__ void scale_kernel(const double* __restrict__ aval, const double* __restrict__ anorm, int64_t nnz,
                             double* __restrict__ E) {
  const double nrm = anorm[0];
  GG_LOOP(e, nnz) E[e] = aval[e] / nrm;
}

__global__ void gather_edge_kernel(const double* __restrict__ X, const double* __restrict__ EI, int de,
                                   double* __restrict__ Z, int fi, const int32_t* __restrict__ rows,
                                   const int32_t* __restrict__ ci, int64_t nnz) {
  GG_LOOP(e, nnz) {
    double* z = Z + e * fi;
    const int64_t r = rows[e], c = ci[e];
    for (int k = 0; k < H; ++k) {
      z[k] = X[r * H + k];
      z[H + k] = X[c * H + k];
    }
    for (int k = 0; k < de; ++k) z[2 * H + k] = EI[e * de + k];
  }
}

__global__ void gather_rows_kernel(const double* __restrict__ Xn, double* __restrict__ Z,
                                   const int32_t* __restrict__ rows, int64_t nnz) {
  GG_LOOP(e, nnz) {
    const int64_t r = rows[e];
    for (int k = 0; k < H; ++k) Z[e * H + k] = Xn[r * H + k];
  }
}

__global__ void fwd_kernel(const Mlp m, const double* __restrict__ Z, int64_t N, double* __restrict__ Y,
                           const double* __restrict__ R) {
  GG_LOOP(k, N) {
    double y[H];
    gg::mlp_fwd(m, Z + k * m.fi, y);
    for (int o = 0; o < m.fo; ++o) Y[k * m.fo + o] = R ? R[k * m.fo + o] + y[o] : y[o];
  }
}

__global__ void bwd_kernel(const Mlp m, const double* __restrict__ Z, const double* __restrict__ DY, int64_t N,
                           double* __restrict__ HID, double* __restrict__ DPRE, double* __restrict__ DZ) {
  GG_LOOP(k, N) gg::mlp_bwd(m, Z + k * m.fi, DY + k * m.fo, HID + k * H, DPRE + k * H, DZ + k * m.fi);
}

__global__ void rowsum_kernel(const double* __restrict__ In, int ld, int off, double* __restrict__ Out, bool zero,
                              const int32_t* __restrict__ rp, int64_t n) {
  GG_LOOP(i, n) {
    for (int c = 0; c < H; ++c) {
      double acc = zero ? 0.0 : Out[i * H + c];
      for (int e = rp[i]; e < rp[i + 1]; ++e) acc += In[(int64_t)e * ld + off + c];
      Out[i * H + c] = acc;
    }
  }
}

__global__ void colsum_kernel(const double* __restrict__ In, int ld, int off, double* __restrict__ Out,
                              const int32_t* __restrict__ rp, const int32_t* __restrict__ inv, int64_t n) {
  GG_LOOP(j, n) {
    for (int c = 0; c < H; ++c) {
      double acc = Out[j * H + c];
      for (int p = rp[j]; p < rp[j + 1]; ++p) acc += In[(int64_t)inv[p] * ld + off + c];
      Out[j * H + c] = acc;
    }
  }
}

__global__ void add_cols_kernel(const double* __restrict__ In, int ld, int off, double* __restrict__ Out,
                                int64_t nnz) {
  GG_LOOP(k, nnz * H) {
    const int64_t e = k / H;
    const int c = (int)(k % H);
    Out[k] += In[e * ld + off + c];
  }
}

// Node graph of a scalar CSR made of dense b x b blocks (block row i: scalar
// rows b i .. b i + b - 1, equal lengths, columns in aligned runs of b):
// block rows start at srp[b i] / b^2; every block's column, its b^2 values
// (row-major) and their scalar positions.  Sets *bad on any other layout.
__global__ void block_graph64_kernel(const int32_t* __restrict__ srp, const int32_t* __restrict__ sci,
                                     const double* __restrict__ aval, int64_t nb, int b, int32_t* __restrict__ brp,
                                     int32_t* __restrict__ bci, double* __restrict__ eraw, int64_t* __restrict__ pos,
                                     int* bad) {
  const int b2 = b * b;
  GG_LOOP(i, nb) {
    const int64_t r0 = (int64_t)b * i;
    const int len = srp[r0 + 1] - srp[r0];
    bool ok = len % b == 0 && srp[r0] % b2 == 0;
    for (int r = 1; ok && r < b; ++r) ok = srp[r0 + r + 1] - srp[r0 + r] == len;
    if (!ok) {
      atomicOr(bad, 1);
      continue;
    }
    const int64_t k0 = srp[r0] / b2;
    brp[i] = (int32_t)k0;
    if (i == nb - 1) brp[nb] = (int32_t)(k0 + len / b);
    for (int q = 0; q < len / b; ++q) {
      const int c0 = sci[srp[r0] + b * q];
      if (c0 % b) atomicOr(bad, 1);
      bci[k0 + q] = c0 / b;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
          const int64_t at = srp[r0 + r] + (int64_t)b * q + c;
          if (sci[at] != c0 + c) atomicOr(bad, 1);
          eraw[(k0 + q) * b2 + r * b + c] = aval[at];
          pos[(k0 + q) * b2 + r * b + c] = at;
        }
    }
  }
}

// inv[position of (j, i) in row j] = the entry (i, j), by binary search in
// row j (columns ascending); sets *bad when the mirror entry is missing.
__global__ void mirror_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const int32_t* __restrict__ rows, int64_t nnz, int32_t* __restrict__ inv, int* bad) {
  GG_LOOP(e, nnz) {
    const int32_t i = rows[e], j = ci[e];
    int lo = rp[j], hi = rp[j + 1] - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ci[mid] < i) lo = mid + 1; else hi = mid;
    }
    if (lo < rp[j + 1] && ci[lo] == i) inv[lo] = (int32_t)e;
    else atomicOr(bad, 1);
  }
}

__global__ void gather_dg_kernel(const double* __restrict__ dG, const int64_t* __restrict__ pos, int64_t count,
                                 double* __restrict__ DY) {
  GG_LOOP(k, count) DY[k] = dG[pos[k]];
}

// Block c: the first-level partial of chunk c for every entry.
__global__ void reduce_partial_kernel(const double* __restrict__ U, int p, const double* __restrict__ V, int q,
                                      int64_t N, double* __restrict__ part) {
  const int P = p * q + p;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * gg::kChunk;
  const int64_t e1 = e0 + gg::kChunk < N ? e0 + gg::kChunk : N;
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) part[c * P + idx] = gg::outer_partial(U, p, V, q, e0, e1, idx);
}

__global__ void reduce_final_kernel(const double* __restrict__ part, int64_t nch, int P, double* __restrict__ dst) {
  GG_LOOP(idx, P) {
    double tot = 0.0;
    for (int64_t c = 0; c < nch; ++c) tot += part[c * P + idx];
    dst[idx] = tot;
  }
}

struct DevOps {
  cudaStream_t s = nullptr;
  int64_t n = 0, nnz = 0;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const int32_t* rows = nullptr;
  const int32_t* inv = nullptr;
  const double* aval = nullptr;     // raw edge features, nnz x b2
  const double* anorm = nullptr;
  const int64_t* pos = nullptr;     // scalar position of every block entry (b2 > 1)
  int b2 = 1;
  std::deque<DevMem> pool;
  int rc = SPAI_OK;

  double* alloc(int64_t count) {
    pool.emplace_back();
    if (int r = pool.back().alloc((size_t)count * sizeof(double), s)) {
      rc = r;
      return nullptr;
    }
    return pool.back().as<double>();
  }
  void zero(double* p, int64_t count) {
    if (cudaMemsetAsync(p, 0, (size_t)count * sizeof(double), s) != cudaSuccess && !rc) rc = SPAI_ERR_CUDA;
  }
  int fail() { return rc ? rc : SPAI_ERR_OOM; }
  int done() {
    if (rc) return rc;
    SPAI_CUDA(cudaGetLastError());
    return SPAI_OK;
  }
  void gather_dg(const double* dG, double* DY) {
    gather_dg_kernel<<<grid_for(nnz * b2), kThreads, 0, s>>>(dG, pos, nnz * b2, DY);
    count_launch();
  }
  void scale_edges(double* E) {
    scale_kernel<<<grid_for(nnz * b2), kThreads, 0, s>>>(aval, anorm, nnz * b2, E);
    count_launch();
  }
  void gather_edge(const double* X, const double* EI, int de, double* Z, int fi) {
    gather_edge_kernel<<<grid_for(nnz), kThreads, 0, s>>>(X, EI, de, Z, fi, rows, ci, nnz);
    count_launch();
  }
  void gather_rows(const double* Xn, double* Z) {
    gather_rows_kernel<<<grid_for(nnz), kThreads, 0, s>>>(Xn, Z, rows, nnz);
    count_launch();
  }
  void fwd(const Mlp& m, const double* Z, int64_t N, double* Y, const double* R) {
    fwd_kernel<<<grid_for(N), kThreads, 0, s>>>(m, Z, N, Y, R);
    count_launch();
  }
  void bwd(const Mlp& m, const double* Z, const double* DY, int64_t N, double* HID, double* DPRE, double* DZ) {
    bwd_kernel<<<grid_for(N), kThreads, 0, s>>>(m, Z, DY, N, HID, DPRE, DZ);
    count_launch();
  }
  void rowsum(const double* In, int ld, int off, double* Out, bool zero_first) {
    rowsum_kernel<<<grid_for(n), kThreads, 0, s>>>(In, ld, off, Out, zero_first, rp, n);
    count_launch();
  }
  void colsum(const double* In, int ld, int off, double* Out) {
    colsum_kernel<<<grid_for(n), kThreads, 0, s>>>(In, ld, off, Out, rp, inv, n);
    count_launch();
  }
  void add_cols(const double* In, int ld, int off, double* Out) {
    add_cols_kernel<<<grid_for(nnz * H), kThreads, 0, s>>>(In, ld, off, Out, nnz);
    count_launch();
  }
  void reduce(const double* U, int p, const double* V, int q, int64_t N, double* dst) {
    const int P = p * q + p;
    const int64_t nch = (N + gg::kChunk - 1) / gg::kChunk;
    pool.emplace_back();
    DevMem& part = pool.back();
    if (int r = part.alloc((size_t)nch * P * sizeof(double), s)) {
      if (!rc) rc = r;
      return;
    }
    reduce_partial_kernel<<<(unsigned)nch, kThreads, 0, s>>>(U, p, V, q, N, part.as<double>());
    count_launch();
    reduce_final_kernel<<<grid_for(P), kThreads, 0, s>>>(part.as<double>(), nch, P, dst);
    count_launch();
  }
};

}  // namespace
}  // namespace spai

using namespace spai;

extern "C" int spai_gnn_grad(const spai_csr* A, const spai_pattern* P, const float* node_feat,
                             const spai_gnn_weights* W, const double* dG, double* dW, void* stream) {
  if (!A || !P || !node_feat || !W || !W->blob || !dG || !dW) return set_error(SPAI_ERR_INVALID, "null argument");
  if (A->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A values must be SPAI_F64");
  const PatternData& Pd = *P->d;
  if (Pd.kind != SPAI_PATTERN_FULL) return set_error(SPAI_ERR_SHAPE, "the GNN writes G on A's full pattern");
  if (Pd.n != A->n || Pd.nnz != A->nnz) return set_error(SPAI_ERR_SHAPE, "pattern was not built from A");
  if (W->d_node < 1 || W->d_node > 16) return set_error(SPAI_ERR_SHAPE, "d_node must be in 1..16");
  if (W->n_layers < 0 || W->n_layers > 8) return set_error(SPAI_ERR_SHAPE, "n_layers must be in 0..8");
  if (W->msg_edge != SPAI_MSG_LATENT && W->msg_edge != SPAI_MSG_RAW) return set_error(SPAI_ERR_INVALID, "msg_edge");
  const int bs = W->block <= 0 ? 1 : W->block;
  if (bs != 1 && bs != 3) return set_error(SPAI_ERR_INVALID, "block size must be 1 or 3");
  if (A->n % bs != 0) return set_error(SPAI_ERR_SHAPE, "n is not a multiple of the block size");
  const int b2 = bs * bs;
  const bool raw = W->msg_edge == SPAI_MSG_RAW;
  const gg::Layout L = gg::make_layout(W->d_node, W->n_layers, raw, b2);
  if (W->count != L.off[L.n_mlp])
    return set_error(SPAI_ERR_SHAPE, "weight blob has %lld floats, layout needs %lld", (long long)W->count,
                     (long long)L.off[L.n_mlp]);
  const int64_t ns = A->n, nnz_s = A->nnz;
  const int64_t n = ns / bs;  // nodes of the graph the GNN runs on
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  DevMem w64, v64, nrm, flag, brp, bci, eraw, pos, idx;
  if ((rc = w64.alloc((size_t)W->count * sizeof(double), s))) return rc;
  if ((rc = v64.alloc((size_t)n * W->d_node * sizeof(double), s))) return rc;
  if ((rc = nrm.alloc(sizeof(double), s))) return rc;
  if ((rc = flag.alloc(sizeof(int), s))) return rc;
  to_f64_kernel<<<grid_for(W->count), kThreads, 0, s>>>(W->blob, W->count, w64.as<double>());
  count_launch();
  to_f64_kernel<<<grid_for(n * W->d_node), kThreads, 0, s>>>(node_feat, n * W->d_node, v64.as<double>());
  count_launch();
  if ((rc = matrix_abs_mean(static_cast<const double*>(A->val), nnz_s, nrm.as<double>(), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  const int32_t* grp = Pd.g_rp();
  const int32_t* gci = Pd.g_ci();
  const double* ev = static_cast<const double*>(A->val);
  int64_t nnz = nnz_s;
  if (bs > 1) {
    // the node graph: at most nnz_s / b2 blocks
    const int64_t cap = nnz_s / b2;
    if ((rc = brp.alloc((size_t)(n + 1) * sizeof(int32_t), s))) return rc;
    if ((rc = bci.alloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t), s))) return rc;
    if ((rc = eraw.alloc((size_t)(cap > 0 ? cap : 1) * b2 * sizeof(double), s))) return rc;
    if ((rc = pos.alloc((size_t)(cap > 0 ? cap : 1) * b2 * sizeof(int64_t), s))) return rc;
    SPAI_CUDA(cudaMemsetAsync(brp.p, 0, (size_t)(n + 1) * sizeof(int32_t), s));
    block_graph64_kernel<<<grid_for(n), kThreads, 0, s>>>(Pd.g_rp(), Pd.g_ci(), ev, n, bs, brp.as<int32_t>(),
                                                          bci.as<int32_t>(), eraw.as<double>(), pos.as<int64_t>(),
                                                          flag.as<int>());
    count_launch();
    int bad = 0;
    SPAI_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    if (bad) return set_error(SPAI_ERR_SHAPE, "A is not made of aligned dense %d x %d blocks", bs, bs);
    nnz = cap;
    grp = brp.as<int32_t>();
    gci = bci.as<int32_t>();
    ev = eraw.as<double>();
  }
  if ((rc = idx.alloc((size_t)2 * (nnz > 0 ? nnz : 1) * sizeof(int32_t), s))) return rc;
  int32_t* rows = idx.as<int32_t>();
  int32_t* inv = rows + nnz;
  rows_kernel<<<grid_for(n), kThreads, 0, s>>>(grp, n, rows);
  count_launch();
  if (bs == 1) {
    inv_kernel<<<grid_for(nnz), kThreads, 0, s>>>(Pd.perm.as<int32_t>(), nnz, inv);
  } else {
    mirror_kernel<<<grid_for(nnz), kThreads, 0, s>>>(grp, gci, rows, nnz, inv, flag.as<int>());
  }
  count_launch();
  if (bs > 1) {
    int bad = 0;
    SPAI_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    if (bad) return set_error(SPAI_ERR_SHAPE, "the block pattern is not symmetric");
  }
  SPAI_CUDA(cudaGetLastError());
  DevOps ops;
  ops.s = s;
  ops.n = n;
  ops.nnz = nnz;
  ops.rp = grp;
  ops.ci = gci;
  ops.rows = rows;
  ops.inv = inv;
  ops.aval = ev;
  ops.anorm = nrm.as<double>();
  ops.b2 = b2;
  ops.pos = bs > 1 ? pos.as<int64_t>() : nullptr;
  return gg::gnn_grad_driver(ops, n, nnz, v64.as<double>(), W->d_node, w64.as<double>(), L, W->n_layers, raw, b2, dG,
                             dW);
}
