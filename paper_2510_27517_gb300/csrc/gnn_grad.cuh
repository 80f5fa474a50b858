// Reverse pass of the GNN (Sec. 3.3 trains the GNN of Sec. 3.2.2, Eqs. 3-5,
// on the SAI loss): from dL/dG on A's pattern to dL/d(every weight), float64.
//
// Written once for two executors: the CUDA kernels of gnn_grad.cu and plain
// host loops (a test harness runs the same driver and element functions on
// the CPU).  Every element function is a fixed sequence of fused
// multiply-adds and every reduction sums in one fixed order, so given the
// same ||A|| both executors give the same bits.
//
// The forward pass is recomputed in float64 with its activations kept (on
// the node graph of the b x b block matrix for b > 1: e is then the block of
// A / ||A|| flattened row-major and D writes a block of G per edge):
//   x_0 = E_n(v),  h_0 = E_e(e),  e = A_ij / ||A||
//   for t < L:  m_t = row sums of f_m(x_t[i], x_t[j], h_t or e)
//               x_{t+1} = x_t + f_v(m_t)
//               h_{t+1} = h_t + f_e(x_{t+1}[i], x_{t+1}[j], h_t)
//   g = D(h_L)
// and walked back: each MLP application turns its output gradient into the
// gradient of its input and the sums over elements of dpre (x) z, dpre,
// dy (x) hid and dy for its weights (dpre = gradient at the hidden layer's
// input, ReLU'(0) = 0).  Scatters to x_i go through the row sums, to x_j
// through the transpose permutation of the pattern (both in entry order).
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define SPAI_GG_HD __host__ __device__
#else
#define SPAI_GG_HD
#endif

namespace spai {
namespace gg {

constexpr int H = 24;             // hidden width (Sec. 4.1)
constexpr int kChunk = 1024;      // elements per first-level weight-gradient partial

// One MLP in float64: W1 (H x fi, row-major), b1 (H), W2 (fo x H), b2 (fo).
struct Mlp {
  const double* w1;
  const double* b1;
  const double* w2;
  const double* b2;
  int fi, fo;
};

SPAI_GG_HD inline double gg_fma(double a, double b, double c) { return fma(a, b, c); }

// y = W2 relu(W1 z + b1) + b2.
SPAI_GG_HD inline void mlp_fwd(const Mlp& p, const double* z, double* y) {
  double hid[H];
  for (int r = 0; r < H; ++r) {
    double a = p.b1[r];
    for (int c = 0; c < p.fi; ++c) a = gg_fma(p.w1[r * p.fi + c], z[c], a);
    hid[r] = a > 0.0 ? a : 0.0;
  }
  for (int o = 0; o < p.fo; ++o) {
    double a = p.b2[o];
    for (int r = 0; r < H; ++r) a = gg_fma(p.w2[o * H + r], hid[r], a);
    y[o] = a;
  }
}

// Reverse pass of one MLP at input z with output gradient dy: the hidden
// activations hid, dpre = (W2^T dy) * [W1 z + b1 > 0] and dz = W1^T dpre.
SPAI_GG_HD inline void mlp_bwd(const Mlp& p, const double* z, const double* dy, double* hid, double* dpre,
                               double* dz) {
  double pre[H];
  for (int r = 0; r < H; ++r) {
    double a = p.b1[r];
    for (int c = 0; c < p.fi; ++c) a = gg_fma(p.w1[r * p.fi + c], z[c], a);
    pre[r] = a;
    hid[r] = a > 0.0 ? a : 0.0;
  }
  for (int r = 0; r < H; ++r) {
    double g = 0.0;
    for (int o = 0; o < p.fo; ++o) g = gg_fma(p.w2[o * H + r], dy[o], g);
    dpre[r] = pre[r] > 0.0 ? g : 0.0;
  }
  for (int c = 0; c < p.fi; ++c) {
    double a = 0.0;
    for (int r = 0; r < H; ++r) a = gg_fma(p.w1[r * p.fi + c], dpre[r], a);
    dz[c] = a;
  }
}

// Entry idx of the first-level partial of elements [e0, e1): for idx < p q
// the (i, j) = (idx / q, idx % q) entry of sum_e U_e V_e^T, else entry
// idx - p q of sum_e U_e.  U is N x p, V is N x q, row-major.
SPAI_GG_HD inline double outer_partial(const double* U, int p, const double* V, int q, int64_t e0, int64_t e1,
                                       int idx) {
  double acc = 0.0;
  if (idx < p * q) {
    const int i = idx / q, j = idx % q;
    for (int64_t e = e0; e < e1; ++e) acc = gg_fma(U[e * p + i], V[e * q + j], acc);
  } else {
    const int i = idx - p * q;
    for (int64_t e = e0; e < e1; ++e) acc += U[e * p + i];
  }
  return acc;
}

// Blob offsets of the MLPs (float counts), in the order E_n, E_e,
// (f_m, f_v, f_e) per layer, D.
struct Layout {
  int n_mlp = 0;
  int fi[2 + 3 * 8 + 1];
  int fo[2 + 3 * 8 + 1];
  int64_t off[2 + 3 * 8 + 2];
};

inline Layout make_layout(int d_node, int n_layers, bool raw, int b2 = 1) {
  Layout L;
  auto add = [&](int fi, int fo) {
    L.fi[L.n_mlp] = fi;
    L.fo[L.n_mlp] = fo;
    L.n_mlp++;
  };
  add(d_node, H);
  add(b2, H);
  for (int t = 0; t < n_layers; ++t) {
    add(2 * H + (raw ? b2 : H), H);
    add(H, H);
    add(3 * H, H);
  }
  add(H, b2);
  L.off[0] = 0;
  for (int k = 0; k < L.n_mlp; ++k)
    L.off[k + 1] = L.off[k] + (int64_t)H * L.fi[k] + H + (int64_t)L.fo[k] * H + L.fo[k];
  return L;
}

inline Mlp mlp_at(const double* w, const Layout& L, int k) {
  Mlp m;
  const double* p = w + L.off[k];
  m.fi = L.fi[k];
  m.fo = L.fo[k];
  m.w1 = p;
  m.b1 = p + (int64_t)H * m.fi;
  m.w2 = m.b1 + H;
  m.b2 = m.w2 + (int64_t)m.fo * H;
  return m;
}

// The driver: one sequence of operations for both executors.  Ops provides
// (arrays live in the executor's memory, float64, row-major):
//   alloc(count) -> double*, zero(p, count), fail() / done() -> status
//   scale_edges(E)                   E[e] = A_e / ||A||, ||A|| = mean |A_e| (Sec. 3.3); b^2 per edge
//   gather_dg(dG, DY)                DY[e][k] = dG at the scalar position of entry k of block edge e
//   gather_edge(X, EI, de, Z, fi)    Z[e] = (X[row e], X[col e], EI[e][0:de]), fi = 2 H + de
//   gather_rows(Xn, Z)               Z[e] = Xn[row e]                      (H wide)
//   fwd(m, Z, N, Y, R)               Y[k] = mlp(Z[k]), plus R[k] when R is given
//   bwd(m, Z, DY, N, HID, DPRE, DZ)  mlp_bwd of every element
//   rowsum(In, ld, off, Out, zero)   Out[i] (=, or +=) sum over row i, in entry order, of In[e][off:off+H]
//   colsum(In, ld, off, Out)         Out[j] += sum over entries (i, j), in entry order, of In[e][off:off+H]
//   add_cols(In, ld, off, Out)       Out[e] += In[e][off:off+H]
//   reduce(U, p, V, q, N, dst)       dst = the outer_partial sums over chunks of kChunk elements,
//                                    chunk partials added in chunk order
// n and nnz count the nodes and edges of the graph the GNN runs on (block
// rows and blocks for b > 1); dG is in the scalar CSR order of G.
template <class Ops>
int gnn_grad_driver(Ops& ops, int64_t n, int64_t nnz, const double* v, int d_node, const double* w,
                    const Layout& L, int n_layers, bool raw, int b2, const double* dG, double* dW) {
  double* E = ops.alloc(nnz * b2);  // e = A / ||A||
  double* DYD = b2 > 1 ? ops.alloc(nnz * b2) : nullptr;
  if (!E || (b2 > 1 && !DYD)) return ops.fail();
  ops.scale_edges(E);
  // activations kept for the reverse pass
  double* X[9];
  double* M[8];
  double* Hs[9];
  for (int t = 0; t <= n_layers; ++t) {
    X[t] = ops.alloc(n * H);
    Hs[t] = ops.alloc(nnz * H);
    if (t < n_layers) M[t] = ops.alloc(n * H);
  }
  const int fim = 2 * H + (raw ? b2 : H);
  double* Z = ops.alloc(nnz * 3 * H);      // inputs of the largest edge MLP
  double* Y = ops.alloc(nnz * H);
  double* HID = ops.alloc(nnz * H);
  double* DPRE = ops.alloc(nnz * H);
  double* DZ = ops.alloc(nnz * 3 * H);
  double* DH = ops.alloc(nnz * H);
  double* DX = ops.alloc(n * H);
  double* DM = ops.alloc(n * H);
  double* DYE = ops.alloc(nnz * H);
  if (!E || !Z || !Y || !HID || !DPRE || !DZ || !DH || !DX || !DM || !DYE) return ops.fail();
  for (int t = 0; t <= n_layers; ++t)
    if (!X[t] || !Hs[t] || (t < n_layers && !M[t])) return ops.fail();

  // ---- forward with activations ----
  ops.fwd(mlp_at(w, L, 0), v, n, X[0], nullptr);
  ops.fwd(mlp_at(w, L, 1), E, nnz, Hs[0], nullptr);
  for (int t = 0; t < n_layers; ++t) {
    const Mlp fm = mlp_at(w, L, 2 + 3 * t), fv = mlp_at(w, L, 3 + 3 * t), fe = mlp_at(w, L, 4 + 3 * t);
    ops.gather_edge(X[t], raw ? E : Hs[t], raw ? b2 : H, Z, fim);
    ops.fwd(fm, Z, nnz, Y, nullptr);
    ops.rowsum(Y, H, 0, M[t], true);
    ops.fwd(fv, M[t], n, X[t + 1], X[t]);
    ops.gather_edge(X[t + 1], Hs[t], H, Z, 3 * H);
    ops.fwd(fe, Z, nnz, Hs[t + 1], Hs[t]);
  }

  // ---- reverse ----
  const int kd = L.n_mlp - 1;
  const Mlp D = mlp_at(w, L, kd);
  const double* DG = dG;
  if (b2 > 1) {
    ops.gather_dg(dG, DYD);
    DG = DYD;
  }
  ops.bwd(D, Hs[n_layers], DG, nnz, HID, DPRE, DH);
  ops.reduce(DPRE, H, Hs[n_layers], H, nnz, dW + L.off[kd]);
  ops.reduce(DG, b2, HID, H, nnz, dW + L.off[kd] + (int64_t)H * H + H);
  ops.zero(DX, n * H);
  for (int t = n_layers - 1; t >= 0; --t) {
    const int km = 2 + 3 * t, kv = 3 + 3 * t, ke = 4 + 3 * t;
    const Mlp fm = mlp_at(w, L, km), fv = mlp_at(w, L, kv), fe = mlp_at(w, L, ke);
    // h_{t+1} = h_t + f_e(x_{t+1}[i], x_{t+1}[j], h_t)
    ops.gather_edge(X[t + 1], Hs[t], H, Z, 3 * H);
    ops.bwd(fe, Z, DH, nnz, HID, DPRE, DZ);
    ops.reduce(DPRE, H, Z, 3 * H, nnz, dW + L.off[ke]);
    ops.reduce(DH, H, HID, H, nnz, dW + L.off[ke] + (int64_t)H * 3 * H + H);
    ops.rowsum(DZ, 3 * H, 0, DX, false);
    ops.colsum(DZ, 3 * H, H, DX);
    ops.add_cols(DZ, 3 * H, 2 * H, DH);
    // x_{t+1} = x_t + f_v(m_t)
    ops.bwd(fv, M[t], DX, n, HID, DPRE, DM);
    ops.reduce(DPRE, H, M[t], H, n, dW + L.off[kv]);
    ops.reduce(DX, H, HID, H, n, dW + L.off[kv] + (int64_t)H * H + H);
    // m_t = row sums of f_m(x_t[i], x_t[j], edge input)
    ops.gather_edge(X[t], raw ? E : Hs[t], raw ? b2 : H, Z, fim);
    ops.gather_rows(DM, DYE);
    ops.bwd(fm, Z, DYE, nnz, HID, DPRE, DZ);
    ops.reduce(DPRE, H, Z, fim, nnz, dW + L.off[km]);
    ops.reduce(DYE, H, HID, H, nnz, dW + L.off[km] + (int64_t)H * fim + H);
    ops.rowsum(DZ, fim, 0, DX, false);
    ops.colsum(DZ, fim, H, DX);
    if (!raw) ops.add_cols(DZ, fim, 2 * H, DH);
  }
  // encoders
  ops.bwd(mlp_at(w, L, 1), E, DH, nnz, HID, DPRE, DZ);
  ops.reduce(DPRE, H, E, b2, nnz, dW + L.off[1]);
  ops.reduce(DH, H, HID, H, nnz, dW + L.off[1] + (int64_t)H * b2 + H);
  ops.bwd(mlp_at(w, L, 0), v, DX, n, HID, DPRE, DZ);
  ops.reduce(DPRE, H, v, d_node, n, dW + L.off[0]);
  ops.reduce(DX, H, HID, H, n, dW + L.off[0] + (int64_t)H * d_node + H);
  return ops.done();
}

}  // namespace gg
}  // namespace spai
