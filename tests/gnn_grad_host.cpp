// Host executor of the GNN reverse-pass driver (paper_2510_27517_gb300/csrc/
// gnn_grad.cuh): the same driver and element functions as the CUDA kernels,
// run as plain loops, so the tests can check them against the oracle on a
// machine without a GPU.  Test infrastructure: built by the tests with g++.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "gnn_grad.cuh"

namespace {

using spai::gg::H;
using spai::gg::Mlp;

struct HostOps {
  int64_t n, nnz;                  // nodes and edges of the graph the GNN runs on
  int b2 = 1;                      // edge feature / decoder width
  const int32_t* rp;
  const int32_t* ci;
  std::vector<double> eraw;        // raw edge features, nnz x b2
  double nrm = 1.0;                // ||A|| over the scalar entries
  std::vector<int64_t> pos;        // scalar position of every block entry, nnz x b2
  std::vector<int32_t> rows, inv;  // row of every entry; entry of every transposed position
  std::vector<std::vector<double>> pool;

  double* alloc(int64_t count) {
    pool.emplace_back((size_t)count, 0.0);
    return pool.back().data();
  }
  void zero(double* p, int64_t count) { std::memset(p, 0, (size_t)count * sizeof(double)); }
  int fail() { return -3; }
  int done() { return 0; }

  void scale_edges(double* E) {
    for (size_t k = 0; k < eraw.size(); ++k) E[k] = eraw[k] / nrm;
  }
  void gather_dg(const double* dG, double* DY) {
    for (size_t k = 0; k < pos.size(); ++k) DY[k] = dG[pos[k]];
  }
  void gather_edge(const double* X, const double* EI, int de, double* Z, int fi) {
    for (int64_t e = 0; e < nnz; ++e) {
      double* z = Z + e * fi;
      for (int c = 0; c < H; ++c) {
        z[c] = X[(int64_t)rows[e] * H + c];
        z[H + c] = X[(int64_t)ci[e] * H + c];
      }
      for (int c = 0; c < de; ++c) z[2 * H + c] = EI[e * de + c];
    }
  }
  void gather_rows(const double* Xn, double* Z) {
    for (int64_t e = 0; e < nnz; ++e)
      for (int c = 0; c < H; ++c) Z[e * H + c] = Xn[(int64_t)rows[e] * H + c];
  }
  void fwd(const Mlp& m, const double* Z, int64_t N, double* Y, const double* R) {
    double y[H];
    for (int64_t k = 0; k < N; ++k) {
      spai::gg::mlp_fwd(m, Z + k * m.fi, y);
      for (int o = 0; o < m.fo; ++o) Y[k * m.fo + o] = R ? R[k * m.fo + o] + y[o] : y[o];
    }
  }
  void bwd(const Mlp& m, const double* Z, const double* DY, int64_t N, double* HID, double* DPRE, double* DZ) {
    for (int64_t k = 0; k < N; ++k)
      spai::gg::mlp_bwd(m, Z + k * m.fi, DY + k * m.fo, HID + k * H, DPRE + k * H, DZ + k * m.fi);
  }
  void rowsum(const double* In, int ld, int off, double* Out, bool zero_first) {
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < H; ++c) {
        double acc = zero_first ? 0.0 : Out[i * H + c];
        for (int e = rp[i]; e < rp[i + 1]; ++e) acc += In[(int64_t)e * ld + off + c];
        Out[i * H + c] = acc;
      }
  }
  void colsum(const double* In, int ld, int off, double* Out) {
    for (int64_t j = 0; j < n; ++j)
      for (int c = 0; c < H; ++c) {
        double acc = Out[j * H + c];
        for (int p = rp[j]; p < rp[j + 1]; ++p) acc += In[(int64_t)inv[p] * ld + off + c];
        Out[j * H + c] = acc;
      }
  }
  void add_cols(const double* In, int ld, int off, double* Out) {
    for (int64_t e = 0; e < nnz; ++e)
      for (int c = 0; c < H; ++c) Out[e * H + c] += In[e * ld + off + c];
  }
  void reduce(const double* U, int p, const double* V, int q, int64_t N, double* dst) {
    const int64_t nch = (N + spai::gg::kChunk - 1) / spai::gg::kChunk;
    for (int idx = 0; idx < p * q + p; ++idx) {
      double tot = 0.0;
      for (int64_t c = 0; c < nch; ++c) {
        const int64_t e0 = c * spai::gg::kChunk, e1 = e0 + spai::gg::kChunk < N ? e0 + spai::gg::kChunk : N;
        tot += spai::gg::outer_partial(U, p, V, q, e0, e1, idx);
      }
      dst[idx] = tot;
    }
  }
};

}  // namespace

// Gradient of sum_e dG[e] G[e] with respect to the weights w (float64 blob in
// the layout of the library's weights), G the GNN's output on the symmetric
// pattern (rowptr, colidx) of A, made of dense b x b blocks when b > 1 (the
// GNN then runs on the node graph of the blocks).  Returns 0, -1 for a
// pattern that is not symmetric or not made of aligned blocks, -2 for
// unsupported sizes.
extern "C" int gnn_grad_host(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* aval,
                             const double* v, int d_node, const double* w, int n_layers, int raw, int b,
                             const double* dG, double* dW) {
  if (n_layers < 0 || n_layers > 8 || d_node < 1 || b < 1 || n % b) return -2;
  HostOps ops;
  const int64_t nnz_s = rowptr[n];
  double sabs = 0.0;
  for (int64_t e = 0; e < nnz_s; ++e) sabs += std::fabs(aval[e]);
  ops.nrm = sabs / (double)nnz_s;
  ops.b2 = b * b;
  std::vector<int32_t> brp, bci;
  if (b == 1) {
    ops.n = n;
    ops.nnz = nnz_s;
    ops.rp = rowptr;
    ops.ci = colidx;
    ops.eraw.assign(aval, aval + nnz_s);
    ops.pos.resize((size_t)nnz_s);
    for (int64_t e = 0; e < nnz_s; ++e) ops.pos[e] = e;
  } else {
    // node graph: block row i lists the blocks of scalar rows b i .. b i + b - 1
    const int64_t nb = n / b;
    brp.assign((size_t)nb + 1, 0);
    for (int64_t i = 0; i < nb; ++i) {
      const int len = rowptr[b * i + 1] - rowptr[b * i];
      if (len % b) return -1;
      for (int r = 1; r < b; ++r)
        if (rowptr[b * i + r + 1] - rowptr[b * i + r] != len) return -1;
      brp[i + 1] = brp[i] + len / b;
    }
    ops.n = nb;
    ops.nnz = brp[nb];
    bci.resize((size_t)ops.nnz);
    ops.eraw.resize((size_t)ops.nnz * ops.b2);
    ops.pos.resize((size_t)ops.nnz * ops.b2);
    for (int64_t i = 0; i < nb; ++i)
      for (int q = 0; q < brp[i + 1] - brp[i]; ++q) {
        const int64_t k = brp[i] + q;
        for (int r = 0; r < b; ++r) {
          const int64_t base = rowptr[b * i + r] + (int64_t)b * q;
          if (colidx[base] % b) return -1;
          if (r == 0) bci[k] = colidx[base] / b;
          else if (colidx[base] / b != bci[k]) return -1;
          for (int c = 0; c < b; ++c) {
            if (colidx[base + c] != colidx[base] + c) return -1;
            ops.eraw[k * ops.b2 + r * b + c] = aval[base + c];
            ops.pos[k * ops.b2 + r * b + c] = base + c;
          }
        }
      }
    ops.rp = brp.data();
    ops.ci = bci.data();
  }
  ops.rows.resize((size_t)ops.nnz);
  ops.inv.assign((size_t)ops.nnz, -1);
  for (int64_t i = 0; i < ops.n; ++i)
    for (int e = ops.rp[i]; e < ops.rp[i + 1]; ++e) ops.rows[e] = (int32_t)i;
  // position of (j, i) in row j for every entry (i, j)
  for (int64_t e = 0; e < ops.nnz; ++e) {
    const int32_t i = ops.rows[e], j = ops.ci[e];
    int p = -1;
    for (int q = ops.rp[j]; q < ops.rp[j + 1]; ++q)
      if (ops.ci[q] == i) p = q;
    if (p < 0) return -1;
    ops.inv[p] = (int32_t)e;
  }
  const spai::gg::Layout L = spai::gg::make_layout(d_node, n_layers, raw != 0, ops.b2);
  return spai::gg::gnn_grad_driver(ops, ops.n, ops.nnz, v, d_node, w, L, n_layers, raw != 0, ops.b2, dG, dW);
}
