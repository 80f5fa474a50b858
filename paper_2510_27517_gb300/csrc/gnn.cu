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

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "gnn_tc.cuh"

namespace spai {

int make_precond_from_values(const std::shared_ptr<PatternData>& P, const void* g_val, int val_dtype, int g_dtype,
                             double eps, std::shared_ptr<PrecondData>& out, cudaStream_t s);

namespace {

constexpr int H = 24;        // hidden width d (Sec. 4.1)
constexpr int MAXD = 16;     // largest node feature width accepted
constexpr int ECAP = 256;    // edges staged per group (= block size)

constexpr int BMAX = 3;      // largest block size b (edge feature and decoder output b^2 wide)
constexpr int B2MAX = BMAX * BMAX;

struct EdgeParams {
  // encoder E_e (first pass only): W1ee is 24 x b^2
  float W1ee[H * B2MAX];
  float b1ee[H];
  float W2ee[H * H];
  float b2ee[H];
  // f_e of this layer (passes t >= 1): h += W2e relu(P_i + Q_j + W1ec h) + b2e
  float W1ec[H * H];
  float W2e[H * H];
  float b2e[H];
  // first layer of the next f_m on the edge input (latent: 24x24, raw: 24 x b^2)
  float W1mc[H * H];
  // decoder D: 24 -> 24 -> b^2
  float W1d[H * H];
  float b1d[H];
  float W2d[B2MAX * H];
  float b2d[B2MAX];
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
  // b x b blocks: the graph above is the node graph; bval holds every block of
  // A / ||A|| (row-major), srp the scalar row pointers G is written through
  const float* bval;
  const int32_t* srp;
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

template <bool FIRST, bool LAST, bool MSG, bool RAW, int B>
__global__ void __launch_bounds__(ECAP) edge_kernel(const EdgeArgs a, const __grid_constant__ EdgeParams w) {
  constexpr int B2 = B * B;
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
          float ev[B2];
          if (B == 1) {
            ev[0] = (float)(__ldg(a.aval + e) / norm);
          } else {
#pragma unroll
            for (int q = 0; q < B2; ++q) ev[q] = __ldg(a.bval + e * B2 + q);
          }
          float h[H];
          if (FIRST) {
            float u[H];
#pragma unroll
            for (int o = 0; o < H; ++o) {
              float acc = w.b1ee[o];
#pragma unroll
              for (int q = 0; q < B2; ++q) acc = fmaf(w.W1ee[o * B2 + q], ev[q], acc);
              u[o] = fmaxf(acc, 0.f);
            }
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
#pragma unroll
                for (int q = 0; q < B2; ++q) acc = fmaf(w.W1mc[o * B2 + q], ev[q], acc);
              } else {
#pragma unroll
                for (int q = 0; q < H; ++q) acc = fmaf(w.W1mc[o * H + q], h[q], acc);
              }
              zbuf[o][k] = fmaxf((pm[o] + qm[o]) + acc, 0.f);
            }
          }
          if (LAST) {
            if (B == 1) {
              float g = 0.f;
#pragma unroll
              for (int o = 0; o < H; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < H; ++q) acc = fmaf(w.W1d[o * H + q], h[q], acc);
                g = fmaf(w.W2d[o], fmaxf(acc + w.b1d[o], 0.f), g);
              }
              g = g + w.b2d[0];
              store_g(a.g_out, a.gtype, e, g);
              store_g(a.gt_out, a.gtype, __ldg(a.perm + e), g);
            } else {
              float hid[H];
#pragma unroll
              for (int o = 0; o < H; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < H; ++q) acc = fmaf(w.W1d[o * H + q], h[q], acc);
                hid[o] = fmaxf(acc + w.b1d[o], 0.f);
              }
              // block e = (block row i, its k-th block): entry (r, c) of G's block
              // sits at scalar position srp[B i + r] + B k + c
              const int64_t k = e - __ldg(a.rp + i);
#pragma unroll
              for (int r = 0; r < B; ++r) {
                const int64_t base = __ldg(a.srp + (int64_t)B * i + r) + (int64_t)B * k;
#pragma unroll
                for (int c = 0; c < B; ++c) {
                  float g = 0.f;
#pragma unroll
                  for (int o = 0; o < H; ++o) g = fmaf(w.W2d[(r * B + c) * H + o], hid[o], g);
                  g = g + w.b2d[r * B + c];
                  store_g(a.g_out, a.gtype, base + c, g);
                  store_g(a.gt_out, a.gtype, __ldg(a.perm + base + c), g);
                }
              }
            }
          }
        }
        if (MSG) {
          __syncthreads();
          if (!longrow) {
            // every (row, channel) sum over the row's edges in edge order, the
            // pairs spread over all threads (channel-major: neighbouring threads
            // take neighbouring rows, whose edges sit in different banks)
            const int nrows = re - r;
            for (int p = threadIdx.x; p < nrows * H; p += blockDim.x) {
              const int c = p / nrows;
              const int row = r + (p - c * nrows);
              const int ea = __ldg(a.rp + row) - cb, eb = __ldg(a.rp + row + 1) - cb;
              float s = 0.f;
              for (int q = ea; q < eb; ++q) s += zbuf[c][q];
              a.S[(int64_t)row * H + c] = s;
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

// ---- per-node MLP layers on the tensor cores (tcgen05, 3xTF32) ----
//
// Weights of one kernel launch live in a device blob prepared on the host:
// for every layer the B operand (N x K, K-major no-swizzle tile) as TF32 hi
// and lo parts, and the bias.  Each block copies the blob to shared memory,
// then walks 128-node tiles: the activations of the tile are written (split
// into hi and lo) as the A operand, one thread issues the MMAs, every thread
// reads its node's row of the accumulator back from tensor memory.
struct TcLayer {
  int K, N;          // padded sizes (K multiple of 8, N multiple of 16)
  int b_hi, b_lo;    // float offsets of the B tiles in the blob
  int bias;          // float offset of the bias (N floats)
};
struct TcNodeParams {
  TcLayer L[5];
  int nlayers;
  int blob_floats;
  int d_node;        // encoder only
  int has_m;
};

constexpr int kTcThreads = tc::kM;

__device__ __forceinline__ void stage_a(float* a_hi, float* a_lo, const float* v, int K) {
  const int row = threadIdx.x;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    if (k < K) {
      const float hi = tc::tf32_rna(v[k]);
      const int off = tc::core_off(row, k, K) >> 2;
      a_hi[off] = hi;
      a_lo[off] = tc::tf32_rna(v[k] - hi);
    }
  }
}

// Issues layer l on A (already staged) and waits; returns false on timeout.
__device__ __forceinline__ bool tc_run_layer(const TcNodeParams& p, int l, const float* blob_s, uint32_t a_hi,
                                             uint32_t a_lo, uint32_t tmem, uint64_t* bar, unsigned& phase,
                                             int* err) {
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
    const TcLayer& L = p.L[l];
    tc::gemm3(tmem, a_hi, a_lo, smem_u32(blob_s + L.b_hi), smem_u32(blob_s + L.b_lo), L.K, L.N);
    tc::mma_commit(bar);
  }
  const bool ok = tc::wait_phase(bar, phase, 2000000000ull);
  phase ^= 1u;
  tc::fence_after_sync();
  if (!ok) atomicExch(err, SPAI_ERR_TIMEOUT);
  return __syncthreads_or(ok ? 0 : 1) == 0;  // every thread leaves together on a timeout
}

// Reads `cnt` (multiple of 16) accumulator columns starting at col0 of this thread's row.
__device__ __forceinline__ void tc_read(uint32_t tmem, int col0, int cnt, float* out) {
  const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) * 32) << 16;
  for (int c = 0; c < cnt; c += 16) tc::tmem_ld16(tmem + lane_base + (uint32_t)(col0 + c), out + c);
}

struct TcSmem {
  float* blob;
  float* a_hi;
  float* a_lo;
  uint32_t tmem;
};

__device__ __forceinline__ void tc_setup(const TcNodeParams& p, const float* __restrict__ blob_g, float* smem,
                                         uint32_t* s_tmem, uint64_t* bar, TcSmem& t) {
  t.a_hi = smem;
  t.a_lo = smem + tc::kM * tc::kKmax;
  t.blob = smem + 2 * tc::kM * tc::kKmax;
  for (int i = threadIdx.x; i < p.blob_floats; i += blockDim.x) t.blob[i] = __ldg(blob_g + i);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(s_tmem)), "n"(tc::kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  t.tmem = *s_tmem;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(tc::kTmemCols) : "memory");
}

__device__ __forceinline__ void store24(float* dst, const float* v) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int k = 0; k < 6; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// x = E_n(v);  PQm = first layer split of f_m of layer 1 (if has_m).
// Layers: 0: relu(v W1^T + b1)  1: * W2^T + b2 (= x)  2: x [Wa;Wb]^T + [b;0]
__global__ void __launch_bounds__(kTcThreads) node_enc_tc_kernel(const float* __restrict__ v, int64_t n, float* x,
                                                                 float* PQm, const float* __restrict__ blob_g,
                                                                 const __grid_constant__ TcNodeParams p, int* err) {
  extern __shared__ __align__(128) float smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  TcSmem t;
  tc_setup(p, blob_g, smem, &s_tmem, &s_bar, t);
  const uint32_t ahi = smem_u32(t.a_hi), alo = smem_u32(t.a_lo);
  unsigned phase = 0;
  const int64_t ntiles = (n + tc::kM - 1) / tc::kM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * tc::kM + threadIdx.x;
    const bool valid = row < n;
    float in[H];
#pragma unroll
    for (int k = 0; k < H; ++k) in[k] = (valid && k < p.d_node) ? __ldg(v + row * p.d_node + k) : 0.f;
    stage_a(t.a_hi, t.a_lo, in, p.L[0].K);
    if (!tc_run_layer(p, 0, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    float d[32];
    tc_read(t.tmem, 0, 32, d);
    float u[H];
#pragma unroll
    for (int o = 0; o < H; ++o) u[o] = fmaxf(d[o] + t.blob[p.L[0].bias + o], 0.f);
    tc::fence_before_sync();
    __syncthreads();
    stage_a(t.a_hi, t.a_lo, u, H);
    if (!tc_run_layer(p, 1, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    tc_read(t.tmem, 0, 32, d);
    float xo[H];
#pragma unroll
    for (int o = 0; o < H; ++o) xo[o] = d[o] + t.blob[p.L[1].bias + o];
    if (valid) store24(x + row * H, xo);
    if (p.has_m) {
      tc::fence_before_sync();
      __syncthreads();
      stage_a(t.a_hi, t.a_lo, xo, H);
      if (!tc_run_layer(p, 2, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
      float pq[48];
      tc_read(t.tmem, 0, 48, pq);
      if (valid) {
        float o48[48];
#pragma unroll
        for (int o = 0; o < 48; ++o) o48[o] = pq[o] + t.blob[p.L[2].bias + o];
        store24(PQm + row * 2 * H, o48);
        store24(PQm + row * 2 * H + H, o48 + H);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  tc_teardown(t.tmem);
}

// One message-passing layer on the nodes:
//   m = W2m S + deg b2m;  x += W2v relu(W1v m + b1v) + b2v;
//   PQe = [Wea;Web] x + [be;0];  PQm = [Wma;Wmb] x + [bm;0] (next layer's f_m)
// Layers: 0: S W2m^T  1: m W1v^T  2: u W2v^T  3: x [Wea;Web;Wma;Wmb]^T
__global__ void __launch_bounds__(kTcThreads) node_layer_tc_kernel(const int32_t* __restrict__ rp, int64_t n,
                                                                   const float* __restrict__ S, float* x, float* PQe,
                                                                   float* PQm, const float* __restrict__ blob_g,
                                                                   const __grid_constant__ TcNodeParams p, int* err) {
  extern __shared__ __align__(128) float smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  TcSmem t;
  tc_setup(p, blob_g, smem, &s_tmem, &s_bar, t);
  const uint32_t ahi = smem_u32(t.a_hi), alo = smem_u32(t.a_lo);
  unsigned phase = 0;
  const int64_t ntiles = (n + tc::kM - 1) / tc::kM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * tc::kM + threadIdx.x;
    const bool valid = row < n;
    float sv[H], xv[H];
    float deg = 0.f;
    if (valid) {
      load24(S + row * H, sv);
      load24(x + row * H, xv);
      deg = (float)(__ldg(rp + row + 1) - __ldg(rp + row));
    } else {
#pragma unroll
      for (int k = 0; k < H; ++k) { sv[k] = 0.f; xv[k] = 0.f; }
    }
    stage_a(t.a_hi, t.a_lo, sv, H);
    if (!tc_run_layer(p, 0, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    float d[32], m[H];
    tc_read(t.tmem, 0, 32, d);
#pragma unroll
    for (int o = 0; o < H; ++o) m[o] = d[o] + deg * t.blob[p.L[0].bias + o];
    tc::fence_before_sync();
    __syncthreads();
    stage_a(t.a_hi, t.a_lo, m, H);
    if (!tc_run_layer(p, 1, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    tc_read(t.tmem, 0, 32, d);
#pragma unroll
    for (int o = 0; o < H; ++o) m[o] = fmaxf(d[o] + t.blob[p.L[1].bias + o], 0.f);
    tc::fence_before_sync();
    __syncthreads();
    stage_a(t.a_hi, t.a_lo, m, H);
    if (!tc_run_layer(p, 2, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    tc_read(t.tmem, 0, 32, d);
#pragma unroll
    for (int o = 0; o < H; ++o) xv[o] = xv[o] + (d[o] + t.blob[p.L[2].bias + o]);
    if (valid) store24(x + row * H, xv);
    tc::fence_before_sync();
    __syncthreads();
    stage_a(t.a_hi, t.a_lo, xv, H);
    if (!tc_run_layer(p, 3, t.blob, ahi, alo, t.tmem, &s_bar, phase, err)) break;
    const int nout = p.L[3].N;  // 48 or 96
    float pq[96];
    tc_read(t.tmem, 0, 48, pq);
    if (nout > 48) tc_read(t.tmem, 48, 48, pq + 48);
    if (valid) {
      float o48[48];
#pragma unroll
      for (int o = 0; o < 48; ++o) o48[o] = pq[o] + t.blob[p.L[3].bias + o];
      store24(PQe + row * 2 * H, o48);
      store24(PQe + row * 2 * H + H, o48 + H);
      if (nout > 48) {
#pragma unroll
        for (int o = 0; o < 48; ++o) o48[o] = pq[48 + o] + t.blob[p.L[3].bias + 48 + o];
        store24(PQm + row * 2 * H, o48);
        store24(PQm + row * 2 * H + H, o48 + H);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  tc_teardown(t.tmem);
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

// TF32 rounding as the device's cvt.rna.tf32.f32: nearest, ties away from zero.
float tf32_host(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// Builds the weight blob of one tensor-core node kernel.
struct TcBlob {
  std::vector<float> f;
  TcNodeParams p;
  TcBlob() { memset(&p, 0, sizeof(p)); }
  // rows[i] = pointer to the K_real inputs of output i (nullptr: zero row);
  // bias[i] (nullptr: zero)
  void add(const std::vector<const float*>& rows, int k_real, const std::vector<float>& bias) {
    const int n_real = (int)rows.size();
    const int N = ((n_real + 15) / 16) * 16, K = ((k_real + 7) / 8) * 8;
    TcLayer& L = p.L[p.nlayers++];
    L.K = K;
    L.N = N;
    L.b_hi = (int)f.size();
    L.b_lo = L.b_hi + N * K;
    L.bias = L.b_lo + N * K;
    f.resize(f.size() + 2 * N * K + N, 0.f);
    for (int r = 0; r < n_real; ++r)
      for (int k = 0; k < k_real; ++k) {
        const float w = rows[r] ? rows[r][k] : 0.f;
        const float hi = tf32_host(w);
        const int off = tc::core_off(r, k, K) >> 2;
        f[L.b_hi + off] = hi;
        f[L.b_lo + off] = tf32_host(w - hi);
      }
    for (int r = 0; r < (int)bias.size() && r < N; ++r) f[L.bias + r] = bias[r];
    p.blob_floats = (int)f.size();
  }
};

struct MLPView {
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  int fi, fo;
};

}  // namespace

namespace {
// Node graph of a scalar CSR made of dense b x b blocks: one thread per block
// row checks that its b scalar rows list the same aligned blocks, and writes
// the block row pointers, block columns and the blocks of A / ||A||.
__global__ void block_graph_kernel(const int32_t* __restrict__ srp, const int32_t* __restrict__ sci,
                                   const double* __restrict__ sval, int64_t nb, int b, const double* __restrict__ norm,
                                   int32_t* browptr, int32_t* bcol, float* bval, int* bad) {
  const double inv = 1.0 / norm[0];
  const int b2 = b * b;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = (int64_t)b * i;
    const int len = srp[r0 + 1] - srp[r0];
    if (len % b != 0 || srp[r0] % b2 != 0) { atomicOr(bad, 1); continue; }
    bool ok = true;
    for (int r = 1; r < b; ++r) ok = ok && (srp[r0 + r + 1] - srp[r0 + r] == len);
    if (!ok) { atomicOr(bad, 1); continue; }
    const int nblk = len / b;
    const int64_t k0 = srp[r0] / b2;
    browptr[i] = (int32_t)k0;
    if (i == nb - 1) browptr[nb] = (int32_t)(k0 + nblk);
    for (int q = 0; q < nblk; ++q) {
      const int c0 = sci[srp[r0] + b * q];
      if (c0 % b != 0) { atomicOr(bad, 1); break; }
      bcol[k0 + q] = c0 / b;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
          const int64_t pos = srp[r0 + r] + (int64_t)b * q + c;
          if (sci[pos] != c0 + c) atomicOr(bad, 1);
          bval[(k0 + q) * b2 + r * b + c] = (float)(sval[pos] * inv);
        }
    }
  }
}
}  // namespace

// ||A|| (Sec. 3.3) into out[0] on the device; the same deterministic sum
// everywhere it is needed.
int matrix_abs_mean(const double* val, int64_t nnz, double* out, cudaStream_t s) {
  const int npart = 4 * num_sms();
  DevMem part;
  int rc;
  if ((rc = part.alloc(sizeof(double) * npart, s))) return rc;
  abs_partial_kernel<<<npart, 256, 0, s>>>(val, nnz, part.as<double>()); count_launch();
  abs_final_kernel<<<1, 256, 0, s>>>(part.as<double>(), npart, nnz, out); count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

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
  const int bs = W->block <= 0 ? 1 : W->block;
  if (bs != 1 && bs != BMAX) return set_error(SPAI_ERR_INVALID, "block size must be 1 or %d", BMAX);
  if (A->n % bs != 0) return set_error(SPAI_ERR_SHAPE, "n is not a multiple of the block size");
  const int b2 = bs * bs;
  const bool raw = W->msg_edge == SPAI_MSG_RAW;
  const int L = W->n_layers, dn = W->d_node;
  // layout (edge feature and decoder output b^2 wide)
  std::vector<std::pair<int, int>> shapes;
  shapes.push_back({dn, H});
  shapes.push_back({b2, H});
  for (int t = 0; t < L; ++t) {
    shapes.push_back({2 * H + (raw ? b2 : H), H});
    shapes.push_back({H, H});
    shapes.push_back({3 * H, H});
  }
  shapes.push_back({H, b2});
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
  auto edge_cols = [&](const MLPView& v, float* dst, int ncol) {
    for (int o = 0; o < H; ++o)
      for (int q = 0; q < ncol; ++q) dst[o * ncol + q] = v.W1[o * v.fi + 2 * H + q];
  };

  const int64_t ns = A->n, nnzs = A->nnz;     // scalar sizes (G's values)
  const int64_t n = ns / bs, nnz = nnzs / b2;   // the GNN's graph: nodes and edges (blocks)
  int rc;
  auto Pre = std::make_shared<PrecondData>();
  Pre->P = P;
  Pre->gtype = g_dtype;
  Pre->eps = eps;
  const size_t es = dtype_size(g_dtype);
  if ((rc = Pre->g_val.alloc((nnzs + 16) * es, s))) return rc;
  if ((rc = Pre->gt_val.alloc((nnzs + 16) * es, s))) return rc;
  Pre->g_val.keep();
  Pre->gt_val.keep();

  // workspace
  const int64_t nnz32 = (nnz + 31) / 32 * 32;
  DevMem hbuf, xbuf, pqe, pqm, sbuf, normb;
  if ((rc = normb.alloc(sizeof(double) * 2, s))) return rc;
  if (L > 0 && (rc = hbuf.alloc((size_t)nnz32 * H * sizeof(float), s))) return rc;
  if ((rc = xbuf.alloc((size_t)n * H * sizeof(float), s))) return rc;
  if ((rc = pqe.alloc((size_t)n * 2 * H * sizeof(float), s))) return rc;
  if ((rc = pqm.alloc((size_t)n * 2 * H * sizeof(float), s))) return rc;
  if ((rc = sbuf.alloc((size_t)n * H * sizeof(float), s))) return rc;

  if ((rc = matrix_abs_mean(static_cast<const double*>(A->val), nnzs, normb.as<double>(), s))) return rc;

  // the graph of the GNN: A's own pattern, or the node graph of its b x b blocks
  const int32_t* grp = P->g_rp();
  const int32_t* gci = P->g_ci();
  DevMem brp, bci, bvl;
  if (bs > 1) {
    DevMem bad;
    if ((rc = brp.alloc((n + 1 + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = bci.alloc((nnz + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = bvl.alloc((nnz * b2 + 16) * sizeof(float), s))) return rc;
    if ((rc = bad.alloc(sizeof(int), s))) return rc;
    SPAI_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    SPAI_CUDA(cudaMemsetAsync(brp.p, 0, (n + 1 + 16) * sizeof(int32_t), s));
    const int bgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    block_graph_kernel<<<bgrid > 0 ? bgrid : 1, 256, 0, s>>>(P->g_rp(), P->g_ci(), static_cast<const double*>(A->val),
                                                             n, bs, normb.as<double>(), brp.as<int32_t>(),
                                                             bci.as<int32_t>(), bvl.as<float>(), bad.as<int>());
    count_launch();
    SPAI_CUDA(cudaGetLastError());
    int hbad = 0;
    SPAI_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    if (hbad) return set_error(SPAI_ERR_BAD_CSR, "A is not made of dense %d x %d blocks", bs, bs);
    grp = brp.as<int32_t>();
    gci = bci.as<int32_t>();
  }

  // tiles of rows for the edge passes
  TileSet et;
  if ((rc = build_tiles(grp, n, nnz, 2048, et, s))) return rc;

  // ---- tensor-core node kernels: launch configuration and weight blobs ----
  const int64_t ntiles = (n + tc::kM - 1) / tc::kM;
  int tgrid = (int)(ntiles < (int64_t)num_sms() * 3 ? ntiles : (int64_t)num_sms() * 3);
  if (tgrid < 1) tgrid = 1;
  DevMem tcerr, encblob;
  if ((rc = tcerr.alloc(sizeof(int), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(tcerr.p, 0, sizeof(int), s));
  auto rows_of = [&](const float* W, int ld, int col0, int nrows) {
    std::vector<const float*> r(nrows);
    for (int i = 0; i < nrows; ++i) r[i] = W + (size_t)i * ld + col0;
    return r;
  };
  auto launch_tc = [&](auto kern, const TcBlob& tb, DevMem& blob, auto... args) -> int {
    int rc2;
    if ((rc2 = blob.alloc(tb.f.size() * sizeof(float), s))) return rc2;
    SPAI_CUDA(cudaMemcpyAsync(blob.p, tb.f.data(), tb.f.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    const size_t smem = (size_t)(2 * tc::kM * tc::kKmax + tb.p.blob_floats) * sizeof(float);
    SPAI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<tgrid, kTcThreads, smem, s>>>(args..., blob.as<float>(), tb.p, tcerr.as<int>());
    count_launch();
    SPAI_CUDA(cudaGetLastError());
    // the blob must stay alive until the kernel ran
    SPAI_CUDA(cudaStreamSynchronize(s));
    return SPAI_OK;
  };
  {
    // x = E_n(v), then the node terms of layer 1's message
    TcBlob tb;
    tb.add(rows_of(En.W1, dn, 0, H), dn, std::vector<float>(En.b1, En.b1 + H));
    tb.add(rows_of(En.W2, H, 0, H), H, std::vector<float>(En.b2, En.b2 + H));
    if (L > 0) {
      const MLPView& m0 = fm(0);
      std::vector<const float*> r = rows_of(m0.W1, m0.fi, 0, H);
      std::vector<const float*> r2 = rows_of(m0.W1, m0.fi, H, H);
      r.insert(r.end(), r2.begin(), r2.end());
      std::vector<float> bias(m0.b1, m0.b1 + H);
      bias.resize(2 * H, 0.f);
      tb.add(r, H, bias);
    }
    tb.p.d_node = dn;
    tb.p.has_m = L > 0;
    if ((rc = launch_tc(node_enc_tc_kernel, tb, encblob, node_feat, n, xbuf.as<float>(), pqm.as<float>()))) return rc;
  }
  EdgeArgs ea;
  memset(&ea, 0, sizeof(ea));
  ea.rp = grp;
  ea.ci = gci;
  ea.aval = static_cast<const double*>(A->val);
  ea.bval = bvl.as<float>();
  ea.srp = P->g_rp();
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
    memcpy(p.W2d, Dd.W2, sizeof(float) * b2 * H);
    memcpy(p.b2d, Dd.b2, sizeof(float) * b2);
  };
  auto fill_msg = [&](EdgeParams& p, int t) {
    if (raw) edge_cols(fm(t), p.W1mc, b2);
    else edge_cols(fm(t), p.W1mc, H);
  };
  // one edge pass, instantiated for the block size
  auto edge_pass = [&](auto first, auto last, auto msg, auto rawc, const EdgeParams& p) -> int {
    constexpr bool F = decltype(first)::value, La = decltype(last)::value, Mg = decltype(msg)::value,
                   Rw = decltype(rawc)::value;
    if (bs == 1) edge_kernel<F, La, Mg, Rw, 1><<<egrid, ECAP, 0, s>>>(ea, p);
    else edge_kernel<F, La, Mg, Rw, BMAX><<<egrid, ECAP, 0, s>>>(ea, p);
    count_launch();
    SPAI_CUDA(cudaGetLastError());
    return SPAI_OK;
  };
  using T = std::true_type;
  using Fl = std::false_type;
  {
    // pass 0: E_e, then the first message (or the decoder when L == 0)
    EdgeParams p;
    memset(&p, 0, sizeof(p));
    for (int o = 0; o < H; ++o) {
      for (int q = 0; q < b2; ++q) p.W1ee[o * b2 + q] = Ee.W1[o * b2 + q];
      p.b1ee[o] = Ee.b1[o];
      p.b2ee[o] = Ee.b2[o];
    }
    memcpy(p.W2ee, Ee.W2, sizeof(p.W2ee));
    if (L == 0) {
      fill_decoder(p);
      rc = edge_pass(T{}, T{}, Fl{}, Fl{}, p);
    } else {
      fill_msg(p, 0);
      rc = raw ? edge_pass(T{}, Fl{}, T{}, T{}, p) : edge_pass(T{}, Fl{}, T{}, Fl{}, p);
    }
    if (rc) return rc;
  }
  for (int t = 0; t < L; ++t) {
    {
      const MLPView& m = fm(t);
      const MLPView& v = fv(t);
      const MLPView& e = fe(t);
      TcBlob tb;
      tb.add(rows_of(m.W2, H, 0, H), H, std::vector<float>(m.b2, m.b2 + H));
      tb.add(rows_of(v.W1, H, 0, H), H, std::vector<float>(v.b1, v.b1 + H));
      tb.add(rows_of(v.W2, H, 0, H), H, std::vector<float>(v.b2, v.b2 + H));
      std::vector<const float*> r = rows_of(e.W1, e.fi, 0, H);
      std::vector<const float*> r2 = rows_of(e.W1, e.fi, H, H);
      r.insert(r.end(), r2.begin(), r2.end());
      std::vector<float> bias(e.b1, e.b1 + H);
      bias.resize(2 * H, 0.f);
      const bool has_m = (t + 1 < L);
      if (has_m) {
        const MLPView& mn = fm(t + 1);
        std::vector<const float*> r3 = rows_of(mn.W1, mn.fi, 0, H);
        std::vector<const float*> r4 = rows_of(mn.W1, mn.fi, H, H);
        r.insert(r.end(), r3.begin(), r3.end());
        r.insert(r.end(), r4.begin(), r4.end());
        bias.insert(bias.end(), mn.b1, mn.b1 + H);
        bias.resize(4 * H, 0.f);
      }
      tb.add(r, H, bias);
      tb.p.has_m = has_m;
      DevMem lblob;
      if ((rc = launch_tc(node_layer_tc_kernel, tb, lblob, grp, n, (const float*)sbuf.as<float>(),
                          xbuf.as<float>(), pqe.as<float>(), pqm.as<float>())))
        return rc;
    }
    EdgeParams p;
    memset(&p, 0, sizeof(p));
    const MLPView& e = fe(t);
    edge_cols(e, p.W1ec, H);
    memcpy(p.W2e, e.W2, sizeof(p.W2e));
    memcpy(p.b2e, e.b2, sizeof(p.b2e));
    if (t + 1 == L) {
      fill_decoder(p);
      rc = edge_pass(Fl{}, T{}, Fl{}, Fl{}, p);
    } else {
      fill_msg(p, t + 1);
      rc = raw ? edge_pass(Fl{}, Fl{}, T{}, T{}, p) : edge_pass(Fl{}, Fl{}, T{}, Fl{}, p);
    }
    if (rc) return rc;
  }
  double hn = 0.0;
  int herr = 0;
  SPAI_CUDA(cudaMemcpyAsync(&hn, normb.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaMemcpyAsync(&herr, tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  if (herr) return set_error(SPAI_ERR_TIMEOUT, "gnn: a tensor-core wait timed out");
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
  if ((rc = precond_sell(*M, (cudaStream_t)stream))) return rc;
  *out = new spai_precond{M};
  return SPAI_OK;
}
