// GNN forward pass that fills G (Sec. 3.2.2, Eqs. 3-5) on A's pattern.
//
//   ||A|| = mean |A_ij| (Sec. 3.3);  e_ij = A_ij / ||A||
//   x_i = E_n(v_i),  h_ij = E_e(e_ij)                         (Eq. 3)
//   for t = 1..L:  m_i = sum_j f_m(x_i, x_j, h_ij)              (Eq. 4)
//                  x_i += f_v(m_i);  h_ij += f_e(x_i, x_j, h_ij)
//   G_ij = D(h_ij)                                             (Eq. 5)
//
// Every MLP is Linear(fan_in -> 24), ReLU, Linear(24 -> fan_out).  The GPU
// evaluates the same functions in a cheaper but equivalent order:
//  * the first linear layer of f_m and f_e acting on the concatenation
//    (x_i, x_j, h_ij) is split as  Wa x_i + Wb x_j + Wc h_ij + b1;  the node
//    terms P_i = Wa x_i + b1 and Q_j = Wb x_j are computed once per node;
//  * the second layer of f_m is linear, so  sum_j (W2 z_ij + b2) =
//    W2 (sum_j z_ij) + deg_i b2: edges only sum z_ij = relu(first layer),
//    and the node kernel applies W2;
//  * each edge pass applies f_e of layer t, then immediately the first layer
//    of f_m of layer t+1 to the updated h (its node terms only need x of
//    layer t, already final), or the decoder D in the last layer.
// Edge work runs on the FP32 FMA pipes with weights in the constant bank
// (kernel parameters): every lane of a warp reads the same weight.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace spai {

int make_precond_from_values(const std::shared_ptr<PatternData>& P, const void* g_val, int val_dtype, int g_dtype,
                             double eps, std::shared_ptr<PrecondData>& out, cudaStream_t s);

namespace {

constexpr int H = 24;        // hidden width d (Sec. 4.1)
constexpr int MAXD = 16;     // largest node feature width accepted
constexpr int ECAP = 256;    // edges staged per group (= block size)

struct PQW {
  float Wa[H * H];
  float Wb[H * H];
  float b[H];
};

struct NodeEncParams {
  float W1[H * MAXD];
  float b1[H];
  float W2[H * H];
  float b2[H];
  PQW m;          // first layer split of f_m of layer 1
  int d_node;
  int has_m;
};

struct NodeLayerParams {
  float W2m[H * H];
  float b2m[H];
  float W1v[H * H];
  float b1v[H];
  float W2v[H * H];
  float b2v[H];
  PQW e;          // f_e of this layer
  PQW m;          // f_m of the next layer
  int has_m;
};

struct EdgeParams {
  // encoder E_e (first pass only)
  float W1ee[H];
  float b1ee[H];
  float W2ee[H * H];
  float b2ee[H];
  // f_e of this layer (passes t >= 1): h += W2e relu(P_i + Q_j + W1ec h) + b2e
  float W1ec[H * H];
  float W2e[H * H];
  float b2e[H];
  // first layer of the next f_m on the edge input (latent: 24x24, raw: 24x1)
  float W1mc[H * H];
  // decoder D
  float W1d[H * H];
  float b1d[H];
  float W2d[H];
  float b2d;
};

struct EdgeArgs {
  const int32_t* rp;
  const int32_t* ci;
  const double* aval;
  const double* anorm;
  const int32_t* tiles;
  int32_t ntiles;
  int64_t nnz;
  float* h;                 // AoSoA [nnz/32][24][32]
  const float* PQe;         // [n][48]  (P | Q) for f_e of this layer
  const float* PQm;         // [n][48]  for f_m of the next layer
  float* S;                 // [n][24]  message sums for the next layer
  void* g_out;              // G values
  void* gt_out;             // G^T values (scattered through perm)
  const int32_t* perm;
  int gtype;
};

__device__ __forceinline__ float* hptr(float* h, int64_t e, int c) {
  return h + ((e >> 5) * (H * 32) + c * 32 + (e & 31));
}

__device__ __forceinline__ void load24(const float* p, float* v) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 t = __ldg(q + k);
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
}

__device__ __forceinline__ void store_g(void* out, int gtype, int64_t i, float v) {
  switch (gtype) {
    case SPAI_F64: static_cast<double*>(out)[i] = (double)v; break;
    case SPAI_F32: static_cast<float*>(out)[i] = v; break;
    case SPAI_BF16: static_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16(v); break;
    default: static_cast<__half*>(out)[i] = __float2half(v); break;
  }
}

template <bool FIRST, bool LAST, bool MSG, bool RAW>
__global__ void __launch_bounds__(ECAP) edge_kernel(const EdgeArgs a, const __grid_constant__ EdgeParams w) {
  __shared__ float zbuf[H][ECAP];
  __shared__ float racc[H];
  const double norm = *a.anorm;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int t0 = __ldg(a.tiles + tile), t1 = __ldg(a.tiles + tile + 1);
    int r = t0;
    while (r < t1) {
      const int base = __ldg(a.rp + r);
      int lo = r, hi = t1;
      while (lo < hi) {
        const int mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(a.rp + mid) - base <= ECAP) lo = mid; else hi = mid - 1;
      }
      const bool longrow = (lo == r);
      const int re = longrow ? r + 1 : lo;
      const int eend = __ldg(a.rp + re);
      if (longrow && threadIdx.x < H) racc[threadIdx.x] = 0.f;
      for (int cb = base; cb < eend; cb += ECAP) {
        const int m = min(ECAP, eend - cb);
        const int k = threadIdx.x;
        if (k < m) {
          const int64_t e = cb + k;
          // row of this edge: last row in [r, re) with rp[row] <= e
          int rl = r, rh = re - 1;
          while (rl < rh) {
            const int mid = rl + ((rh - rl + 1) >> 1);
            if (__ldg(a.rp + mid) <= e) rl = mid; else rh = mid - 1;
          }
          const int i = rl;
          const int j = __ldg(a.ci + e);
          const float ev = (float)(__ldg(a.aval + e) / norm);
          float h[H];
          if (FIRST) {
            float u[H];
#pragma unroll
            for (int o = 0; o < H; ++o) u[o] = fmaxf(fmaf(w.W1ee[o], ev, w.b1ee[o]), 0.f);
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = 0.f;
#pragma unroll
              for (int q = 0; q < H; ++q) acc = fmaf(w.W2ee[o * H + q], u[q], acc);
              h[o] = acc + w.b2ee[o];
            }
          } else {
#pragma unroll
            for (int c = 0; c < H; ++c) h[c] = *hptr(a.h, e, c);
            float pe[H], qe[H], u[H];
            load24(a.PQe + (int64_t)i * 2 * H, pe);
            load24(a.PQe + (int64_t)j * 2 * H + H, qe);
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = 0.f;
#pragma unroll
              for (int q = 0; q < H; ++q) acc = fmaf(w.W1ec[o * H + q], h[q], acc);
              u[o] = fmaxf((pe[o] + qe[o]) + acc, 0.f);
            }
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = 0.f;
#pragma unroll
              for (int q = 0; q < H; ++q) acc = fmaf(w.W2e[o * H + q], u[q], acc);
              h[o] = h[o] + (acc + w.b2e[o]);
            }
          }
          if (!LAST) {
#pragma unroll
            for (int c = 0; c < H; ++c) *hptr(a.h, e, c) = h[c];
          }
          if (MSG) {
            float pm[H], qm[H];
            load24(a.PQm + (int64_t)i * 2 * H, pm);
            load24(a.PQm + (int64_t)j * 2 * H + H, qm);
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = 0.f;
              if (RAW) {
                acc = w.W1mc[o] * ev;
              } else {
#pragma unroll
                for (int q = 0; q < H; ++q) acc = fmaf(w.W1mc[o * H + q], h[q], acc);
              }
              zbuf[o][k] = fmaxf((pm[o] + qm[o]) + acc, 0.f);
            }
          }
          if (LAST) {
            float g = 0.f;
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = 0.f;
#pragma unroll
              for (int q = 0; q < H; ++q) acc = fmaf(w.W1d[o * H + q], h[q], acc);
              g = fmaf(w.W2d[o], fmaxf(acc + w.b1d[o], 0.f), g);
            }
            g = g + w.b2d;
            store_g(a.g_out, a.gtype, e, g);
            store_g(a.gt_out, a.gtype, __ldg(a.perm + e), g);
          }
        }
        if (MSG) {
          __syncthreads();
          if (!longrow) {
            for (int row = r + threadIdx.x; row < re; row += blockDim.x) {
              const int ea = __ldg(a.rp + row) - cb, eb = __ldg(a.rp + row + 1) - cb;
              float* out = a.S + (int64_t)row * H;
#pragma unroll 4
              for (int c = 0; c < H; ++c) {
                float s = 0.f;
                for (int q = ea; q < eb; ++q) s += zbuf[c][q];
                out[c] = s;
              }
            }
          } else if (threadIdx.x < H) {
            float s = racc[threadIdx.x];
            for (int q = 0; q < m; ++q) s += zbuf[threadIdx.x][q];
            racc[threadIdx.x] = s;
          }
          __syncthreads();
        }
      }
      if (MSG && longrow && threadIdx.x < H) a.S[(int64_t)r * H + threadIdx.x] = racc[threadIdx.x];
      __syncthreads();
      r = re;
    }
  }
}

__device__ __forceinline__ void pq_store(const PQW& p, const float* x, float* out) {
#pragma unroll
  for (int o = 0; o < H; ++o) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int q = 0; q < H; ++q) {
      a = fmaf(p.Wa[o * H + q], x[q], a);
      b = fmaf(p.Wb[o * H + q], x[q], b);
    }
    out[o] = a + p.b[o];
    out[H + o] = b;
  }
}

__global__ void __launch_bounds__(128) node_enc_kernel(const float* __restrict__ v, int64_t n, float* x,
                                                       float* PQm, const __grid_constant__ NodeEncParams w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float in[MAXD];
#pragma unroll
    for (int k = 0; k < MAXD; ++k) in[k] = (k < w.d_node) ? __ldg(v + i * w.d_node + k) : 0.f;
    float u[H], xo[H];
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < MAXD; ++k) acc = fmaf(w.W1[o * MAXD + k], in[k], acc);
      u[o] = fmaxf(acc + w.b1[o], 0.f);
    }
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < H; ++q) acc = fmaf(w.W2[o * H + q], u[q], acc);
      xo[o] = acc + w.b2[o];
    }
    float4* xp = reinterpret_cast<float4*>(x + i * H);
#pragma unroll
    for (int k = 0; k < 6; ++k) xp[k] = make_float4(xo[4 * k], xo[4 * k + 1], xo[4 * k + 2], xo[4 * k + 3]);
    if (w.has_m) {
      float pq[2 * H];
      pq_store(w.m, xo, pq);
      float4* pp = reinterpret_cast<float4*>(PQm + i * 2 * H);
#pragma unroll
      for (int k = 0; k < 12; ++k) pp[k] = make_float4(pq[4 * k], pq[4 * k + 1], pq[4 * k + 2], pq[4 * k + 3]);
    }
  }
}

__global__ void __launch_bounds__(128) node_layer_kernel(const int32_t* __restrict__ rp, int64_t n,
                                                         const float* __restrict__ S, float* x, float* PQe,
                                                         float* PQm, const __grid_constant__ NodeLayerParams w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float deg = (float)(__ldg(rp + i + 1) - __ldg(rp + i));
    float s[H], m[H], u[H], xv[H];
    load24(S + i * H, s);
    load24(x + i * H, xv);
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < H; ++q) acc = fmaf(w.W2m[o * H + q], s[q], acc);
      m[o] = acc + deg * w.b2m[o];
    }
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < H; ++q) acc = fmaf(w.W1v[o * H + q], m[q], acc);
      u[o] = fmaxf(acc + w.b1v[o], 0.f);
    }
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < H; ++q) acc = fmaf(w.W2v[o * H + q], u[q], acc);
      xv[o] = xv[o] + (acc + w.b2v[o]);
    }
    float4* xp = reinterpret_cast<float4*>(x + i * H);
#pragma unroll
    for (int k = 0; k < 6; ++k) xp[k] = make_float4(xv[4 * k], xv[4 * k + 1], xv[4 * k + 2], xv[4 * k + 3]);
    float pq[2 * H];
    pq_store(w.e, xv, pq);
    float4* pe = reinterpret_cast<float4*>(PQe + i * 2 * H);
#pragma unroll
    for (int k = 0; k < 12; ++k) pe[k] = make_float4(pq[4 * k], pq[4 * k + 1], pq[4 * k + 2], pq[4 * k + 3]);
    if (w.has_m) {
      pq_store(w.m, xv, pq);
      float4* pm = reinterpret_cast<float4*>(PQm + i * 2 * H);
#pragma unroll
      for (int k = 0; k < 12; ++k) pm[k] = make_float4(pq[4 * k], pq[4 * k + 1], pq[4 * k + 2], pq[4 * k + 3]);
    }
  }
}

// ||A|| = mean |A_ij| in float64, deterministic two-level sum.
__global__ void abs_partial_kernel(const double* __restrict__ v, int64_t m, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    s += fabs(v[i]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void abs_final_kernel(const double* part, int np, int64_t m, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = s / (double)m;
}

struct MLPView {
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  int fi, fo;
};

}  // namespace

int gnn_forward(const spai_csr* A, const std::shared_ptr<PatternData>& P, const float* node_feat,
                const spai_gnn_weights* W, int g_dtype, double eps, std::shared_ptr<PrecondData>& out,
                cudaStream_t s) {
  if (!A || !node_feat || !W || !W->blob) return set_error(SPAI_ERR_INVALID, "null argument");
  if (A->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A values must be SPAI_F64");
  if (P->kind != SPAI_PATTERN_FULL) return set_error(SPAI_ERR_SHAPE, "the GNN writes G on A's full pattern");
  if (P->n != A->n || P->nnz != A->nnz) return set_error(SPAI_ERR_SHAPE, "pattern was not built from A");
  if (W->d_node < 1 || W->d_node > MAXD) return set_error(SPAI_ERR_SHAPE, "d_node must be in 1..%d", MAXD);
  if (W->n_layers < 0 || W->n_layers > 8) return set_error(SPAI_ERR_SHAPE, "n_layers must be in 0..8");
  if (W->msg_edge != SPAI_MSG_LATENT && W->msg_edge != SPAI_MSG_RAW) return set_error(SPAI_ERR_INVALID, "msg_edge");
  if (!dtype_size(g_dtype)) return set_error(SPAI_ERR_INVALID, "unknown G dtype");
  const bool raw = W->msg_edge == SPAI_MSG_RAW;
  const int L = W->n_layers, dn = W->d_node;
  // layout
  std::vector<std::pair<int, int>> shapes;
  shapes.push_back({dn, H});
  shapes.push_back({1, H});
  for (int t = 0; t < L; ++t) {
    shapes.push_back({2 * H + (raw ? 1 : H), H});
    shapes.push_back({H, H});
    shapes.push_back({3 * H, H});
  }
  shapes.push_back({H, 1});
  int64_t need = 0;
  for (auto& sh : shapes) need += (int64_t)H * sh.first + H + (int64_t)sh.second * H + sh.second;
  if (W->count != need)
    return set_error(SPAI_ERR_SHAPE, "weight blob has %lld floats, layout needs %lld", (long long)W->count,
                     (long long)need);
  std::vector<float> hw(need);
  SPAI_CUDA(cudaMemcpyAsync(hw.data(), W->blob, need * sizeof(float), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  std::vector<MLPView> mv;
  {
    int64_t o = 0;
    for (auto& sh : shapes) {
      MLPView v;
      v.fi = sh.first;
      v.fo = sh.second;
      v.W1 = hw.data() + o; o += (int64_t)H * v.fi;
      v.b1 = hw.data() + o; o += H;
      v.W2 = hw.data() + o; o += (int64_t)v.fo * H;
      v.b2 = hw.data() + o; o += v.fo;
      mv.push_back(v);
    }
  }
  const MLPView& En = mv[0];
  const MLPView& Ee = mv[1];
  const MLPView& Dd = mv.back();
  auto fm = [&](int t) -> const MLPView& { return mv[2 + 3 * t]; };
  auto fv = [&](int t) -> const MLPView& { return mv[3 + 3 * t]; };
  auto fe = [&](int t) -> const MLPView& { return mv[4 + 3 * t]; };
  auto split = [&](const MLPView& v, PQW& p) {
    for (int o = 0; o < H; ++o)
      for (int q = 0; q < H; ++q) {
        p.Wa[o * H + q] = v.W1[o * v.fi + q];
        p.Wb[o * H + q] = v.W1[o * v.fi + H + q];
      }
    for (int o = 0; o < H; ++o) p.b[o] = v.b1[o];
  };
  auto edge_cols = [&](const MLPView& v, float* dst, int ncol) {
    for (int o = 0; o < H; ++o)
      for (int q = 0; q < ncol; ++q) dst[o * ncol + q] = v.W1[o * v.fi + 2 * H + q];
  };

  const int64_t n = A->n, nnz = A->nnz;
  int rc;
  auto Pre = std::make_shared<PrecondData>();
  Pre->P = P;
  Pre->gtype = g_dtype;
  Pre->eps = eps;
  const size_t es = dtype_size(g_dtype);
  if ((rc = Pre->g_val.alloc((nnz + 16) * es, s))) return rc;
  if ((rc = Pre->gt_val.alloc((nnz + 16) * es, s))) return rc;
  Pre->g_val.keep();
  Pre->gt_val.keep();

  // workspace
  const int64_t nnz32 = (nnz + 31) / 32 * 32;
  DevMem hbuf, xbuf, pqe, pqm, sbuf, normb, part;
  const int npart = 4 * num_sms();
  if ((rc = normb.alloc(sizeof(double) * 2, s))) return rc;
  if ((rc = part.alloc(sizeof(double) * npart, s))) return rc;
  if (L > 0 && (rc = hbuf.alloc((size_t)nnz32 * H * sizeof(float), s))) return rc;
  if ((rc = xbuf.alloc((size_t)n * H * sizeof(float), s))) return rc;
  if ((rc = pqe.alloc((size_t)n * 2 * H * sizeof(float), s))) return rc;
  if ((rc = pqm.alloc((size_t)n * 2 * H * sizeof(float), s))) return rc;
  if ((rc = sbuf.alloc((size_t)n * H * sizeof(float), s))) return rc;

  abs_partial_kernel<<<npart, 256, 0, s>>>(static_cast<const double*>(A->val), nnz, part.as<double>()); count_launch();
  abs_final_kernel<<<1, 256, 0, s>>>(part.as<double>(), npart, nnz, normb.as<double>()); count_launch();
  SPAI_CUDA(cudaGetLastError());

  // tiles of rows for the edge passes
  TileSet et;
  if ((rc = build_tiles(P->g_rp(), n, nnz, 2048, et, s))) return rc;

  const int nb = 128;
  int ngrid = (int)((n + nb - 1) / nb);
  if (ngrid > num_sms() * 32) ngrid = num_sms() * 32;
  {
    NodeEncParams p;
    memset(&p, 0, sizeof(p));
    for (int o = 0; o < H; ++o)
      for (int k = 0; k < dn; ++k) p.W1[o * MAXD + k] = En.W1[o * dn + k];
    memcpy(p.b1, En.b1, sizeof(p.b1));
    memcpy(p.W2, En.W2, sizeof(p.W2));
    memcpy(p.b2, En.b2, sizeof(p.b2));
    p.d_node = dn;
    p.has_m = L > 0;
    if (L > 0) split(fm(0), p.m);
    node_enc_kernel<<<ngrid, nb, 0, s>>>(node_feat, n, xbuf.as<float>(), pqm.as<float>(), p); count_launch();
    SPAI_CUDA(cudaGetLastError());
  }
  EdgeArgs ea;
  memset(&ea, 0, sizeof(ea));
  ea.rp = P->g_rp();
  ea.ci = P->g_ci();
  ea.aval = static_cast<const double*>(A->val);
  ea.anorm = normb.as<double>();
  ea.tiles = et.starts.as<int32_t>();
  ea.ntiles = et.ntiles;
  ea.nnz = nnz;
  ea.h = hbuf.as<float>();
  ea.PQe = pqe.as<float>();
  ea.PQm = pqm.as<float>();
  ea.S = sbuf.as<float>();
  ea.g_out = Pre->g_val.p;
  ea.gt_out = Pre->gt_val.p;
  ea.perm = P->perm.as<int32_t>();
  ea.gtype = g_dtype;
  int egrid = et.ntiles;
  if (egrid > num_sms() * 8) egrid = num_sms() * 8;
  auto fill_decoder = [&](EdgeParams& p) {
    memcpy(p.W1d, Dd.W1, sizeof(p.W1d));
    memcpy(p.b1d, Dd.b1, sizeof(p.b1d));
    memcpy(p.W2d, Dd.W2, sizeof(p.W2d));
    p.b2d = Dd.b2[0];
  };
  auto fill_msg = [&](EdgeParams& p, int t) {
    if (raw) edge_cols(fm(t), p.W1mc, 1);
    else edge_cols(fm(t), p.W1mc, H);
  };
  {
    // pass 0: E_e, then the first message (or the decoder when L == 0)
    EdgeParams p;
    memset(&p, 0, sizeof(p));
    for (int o = 0; o < H; ++o) { p.W1ee[o] = Ee.W1[o]; p.b1ee[o] = Ee.b1[o]; p.b2ee[o] = Ee.b2[o]; }
    memcpy(p.W2ee, Ee.W2, sizeof(p.W2ee));
    if (L == 0) {
      fill_decoder(p);
      edge_kernel<true, true, false, false><<<egrid, ECAP, 0, s>>>(ea, p); count_launch();
    } else {
      fill_msg(p, 0);
      if (raw) { edge_kernel<true, false, true, true><<<egrid, ECAP, 0, s>>>(ea, p); count_launch(); }
      else { edge_kernel<true, false, true, false><<<egrid, ECAP, 0, s>>>(ea, p); count_launch(); }
    }
    SPAI_CUDA(cudaGetLastError());
  }
  for (int t = 0; t < L; ++t) {
    NodeLayerParams np_;
    memset(&np_, 0, sizeof(np_));
    const MLPView& m = fm(t);
    const MLPView& v = fv(t);
    memcpy(np_.W2m, m.W2, sizeof(np_.W2m));
    memcpy(np_.b2m, m.b2, sizeof(np_.b2m));
    memcpy(np_.W1v, v.W1, sizeof(np_.W1v));
    memcpy(np_.b1v, v.b1, sizeof(np_.b1v));
    memcpy(np_.W2v, v.W2, sizeof(np_.W2v));
    memcpy(np_.b2v, v.b2, sizeof(np_.b2v));
    split(fe(t), np_.e);
    np_.has_m = (t + 1 < L);
    if (np_.has_m) split(fm(t + 1), np_.m);
    node_layer_kernel<<<ngrid, nb, 0, s>>>(P->g_rp(), n, sbuf.as<float>(), xbuf.as<float>(), pqe.as<float>(),
                                           pqm.as<float>(), np_); count_launch();
    SPAI_CUDA(cudaGetLastError());
    EdgeParams p;
    memset(&p, 0, sizeof(p));
    const MLPView& e = fe(t);
    edge_cols(e, p.W1ec, H);
    memcpy(p.W2e, e.W2, sizeof(p.W2e));
    memcpy(p.b2e, e.b2, sizeof(p.b2e));
    if (t + 1 == L) {
      fill_decoder(p);
      edge_kernel<false, true, false, false><<<egrid, ECAP, 0, s>>>(ea, p); count_launch();
    } else {
      fill_msg(p, t + 1);
      if (raw) { edge_kernel<false, false, true, true><<<egrid, ECAP, 0, s>>>(ea, p); count_launch(); }
      else { edge_kernel<false, false, true, false><<<egrid, ECAP, 0, s>>>(ea, p); count_launch(); }
    }
    SPAI_CUDA(cudaGetLastError());
  }
  double hn = 0.0;
  SPAI_CUDA(cudaMemcpyAsync(&hn, normb.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  Pre->anorm = hn;
  out = Pre;
  return SPAI_OK;
}

}  // namespace spai

using namespace spai;

extern "C" int spai_gnn_precond(const spai_csr* A, const spai_pattern* P, const float* node_feat,
                                const spai_gnn_weights* W, int32_t g_dtype, double eps, spai_precond** out,
                                void* stream) {
  if (!out || !P) return set_error(SPAI_ERR_INVALID, "null argument");
  *out = nullptr;
  if (!(eps >= 0.0)) return set_error(SPAI_ERR_INVALID, "eps must be >= 0");
  std::shared_ptr<PrecondData> M;
  int rc = gnn_forward(A, P->d, node_feat, W, g_dtype, eps, M, (cudaStream_t)stream);
  if (rc) return rc;
  *out = new spai_precond{M};
  return SPAI_OK;
}
