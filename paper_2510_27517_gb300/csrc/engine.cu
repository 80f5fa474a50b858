// Persistent preconditioned-CG engine.
//
// Algorithm 1 (App. A) with M^-1 = G G^T + eps I (Eq. 1) applied as two row
// gathers (Eq. 2: first t = G^T r over the explicit transposed CSR, then
// s = G t + eps r).  One cooperative kernel runs many iterations (and many
// independent systems) without returning to the host: every system carries a
// small state machine, and the kernel advances all live systems by one
// "phase" per grid-wide step.  A phase is one pass over one sparse matrix
// (A, G^T or G) plus the vector updates that can ride along with it:
//
//   P1      p = s + beta d  (p = s on the first step),  d' = p,  q = A p,  p.q
//   P2      x += alpha d,  r' = r - alpha q,  t = G^T r',  r'.r'
//   APPLY2  s = G t + eps r,  r.s            (beta = delta_new / delta_old next)
//   RESID   r = b - A x (true residual: every `period` iterations and to
//           confirm convergence), r.r
//   APPLY1  t = G^T r after a RESID
//
// so a regular iteration costs three passes and three grid barriers.  Row
// sums accumulate entry by entry in stored order with fused multiply-adds, and
// the vector updates a + b*c are single fused multiply-adds (one rounding each:
// on this GPU float64 instructions are scarce, and fusing halves them); values
// that are both stored and recomputed on the fly (r', p) use the same
// expression, so every block sees bit-identical values.
//
// Mixed precision (SPAI_PREC_MIXED): the same iteration runs on float32 A, G
// and vectors with float64 dot products; it solves A e = r64 to a relative
// tolerance, then the float64 outer step x += e, r64 = b - A x (float64 SpMV)
// restarts it until ||r64|| <= rtol ||b||.
//
// Reductions: every tile writes its partial sums; the block that finishes
// the last tile of a system for the current phase sums that system's tile
// partials in a fixed order and computes the system's next state.  Results
// therefore depend only on the system and its schedule, not on the other
// systems in the launch or on which block ran which tile.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "deal.h"
#include "internal.cuh"

namespace spai {

namespace {

enum Phase : int32_t {
  PH_RESID0 = 0, PH_APPLY1, PH_APPLY2, PH_P1, PH_P2, PH_P2X, PH_RESID, PH_XUPD, PH_RESID64, PH_ZEROX, PH_P2F, PH_DONE
};
enum Mat : int { MAT_A = 0, MAT_GT = 1, MAT_G = 2 };

__host__ __device__ inline int phase_mat(int ph) {
  return (ph == PH_APPLY1 || ph == PH_P2) ? MAT_GT : (ph == PH_APPLY2 ? MAT_G : MAT_A);
}

struct EngSys {
  const int32_t* rp[3];
  const int32_t* ci[3];
  const void* val[3];     // A (float64 or float32 by mode), G^T, G (G's storage type)
  const double* a_v64;    // float64 values of A (outer residual in mixed mode)
  const int32_t* tiles[3];  // group row starts per matrix
  int32_t ntiles[3];        // groups per matrix
  int32_t kgroups[3];       // groups per work item per matrix
  int32_t fits[3];          // every group fits the stage buffer
  int32_t fmt[3];           // 0: CSR row groups (tiles = rows), 1: SELL-32 (tiles = slices),
                            // 2: 3 x 3 blocks (tiles = slices of 32 block rows)
  const int32_t* sptr[3];   // SELL-32 slice offsets (fmt 1)
  const int32_t* srow[3];   // SELL-32 row at every slice position (rows sorted by length), or nullptr
  const int32_t* a_ci64;    // CSR column indices of A (float64 residual of mixed mode)
  int32_t nitems;           // work items of this system
  int32_t item_base;
  int32_t chunk_base;     // first chunk counter / chunk partial of this system
  int32_t fuse;           // 1: the G^T and G passes share one grid step (PH_P2F), ordered by item flags
  const int32_t* dep;     // fuse: per item, the first and last G^T-pass items whose rows its G rows reach
  int32_t pair;           // 1: s with d and q with r stored as interleaved pairs (r[k], d[k] point at the
                          // odd elements; q and s unused); kernel variants 1 and 2 only
  int64_t n;
  double eps;
  const double* b;
  double* x;
  void* r[2];
  void* d[2];
  void* q;
  void* t;
  void* s;
  void* e;
  void* rin;
  double* history;
  int64_t history_len;
  double* lanczos;
  int64_t lanczos_len;
};

struct EngOpts {
  double tol2;
  double reliable2;   // mixed: replace when ||r||^2 <= reliable2 * ||r_ref||^2
  int64_t max_iter;
  int32_t period, criterion, max_outer, mixed;
};

struct __align__(16) EngState {
  int32_t phase, status, rc, dc;
  int32_t first, first_resid, outer, e_dirty;
  int32_t stop, stop_ok, pad0, pad1;
  int64_t iter, hist_n;
  double delta, delta0, alpha, beta, bb, rr, rr_ref, pad2;
};
static_assert(sizeof(EngState) % 8 == 0, "state words");

struct EngArgs {
  const EngSys* sys;
  EngState* st0;
  EngState* st1;
  int32_t nsys;
  const int32_t* item_sys;
  const int32_t* item_tile;
  int32_t n_items;
  double* partial;        // per tile: 2 doubles
  double* cpartial;       // per chunk of kChunk tiles: 2 doubles
  unsigned* cnt;          // per system: chunks completed in this slot
  unsigned* ccnt;         // per chunk: tiles completed in this slot
  GridSync* gs;
  unsigned* flags;        // per item: the grid step (+1) in which its G^T pass of a fused step completed
  EngOpts o;
  int32_t max_slots;
  int32_t cap;  // staging capacity in entries
  uint64_t limit_ns;
};

template <class T> struct Conv;
template <> struct Conv<double> {
  template <class U> __device__ static double f(U v) { return to_f64(v); }
};
template <> struct Conv<float> {
  template <class U> __device__ static float f(U v) { return to_f32(v); }
};

constexpr int kBlock = 256;   // threads per block
constexpr int kNE = 8;        // staged entries per thread per group
constexpr int kCap = kNE * kBlock;
constexpr int kChunk = 32;    // items per first-level reduction chunk
constexpr int kStages32 = 3;  // TMA stage ring depth of CSR groups (float32 kernels)
constexpr int kStagesSell32 = 3;  // ring depth of SELL-32 groups (float32 kernels)
constexpr int kStages64 = 2;  // TMA stage ring depth (float64 kernels)
constexpr int kStages = 4;    // largest ring (shared-memory arrays)
constexpr int kMaxK = 64;     // groups per work item at most
constexpr int kWarpE = 256;   // entries per warp product chunk
constexpr int kAlignE = 8;    // bulk copies start at multiples of 8 entries (16 B for every type)
constexpr int kSlicesInReg = 63;  // SELL groups of up to this many slices keep their offsets in registers
// GridSync::err value of a launch-table entry out of range (never expected:
// the kernel skips the entry and the host reports it).
constexpr int kErrTable = -100;

// y_row = sum over the row's entries of val * op.gather(col), in stored
// order, then op.fin(row, y_row, op.pre(row)).  Rows are processed in groups
// whose entries fit kCap: every thread first issues all of its entry loads
// (column, value) and all gathers, stores the products in shared memory, then
// issues the operand loads of its rows (op.pre) before summing.  A row with
// more than kCap entries is summed by the whole block (fixed tree).
template <class AT, class MV, class Op>
__device__ __forceinline__ void spmv_group(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                           const MV* __restrict__ val, int r, int re, int base, int m, AT* sbuf,
                                           const Op& op, double& p0, double& p1, uint32_t& blocks) {
  {
    int cix[kNE];
    AT v[kNE];
#pragma unroll
    for (int u = 0; u < kNE; ++u) {
      const int k = threadIdx.x + u * kBlock;
      cix[u] = (k < m) ? __ldg(ci + base + k) : 0;
      v[u] = (k < m) ? Conv<AT>::f(ldro(val + base + k)) : AT(0);
    }
    AT g[kNE];
#pragma unroll
    for (int u = 0; u < kNE; ++u) {
      const int k = threadIdx.x + u * kBlock;
      g[u] = (k < m) ? op.gather(cix[u]) : AT(0);
    }
#pragma unroll
    for (int u = 0; u < kNE; ++u) {
      const int k = threadIdx.x + u * kBlock;
      if (k < m) sbuf[k] = g[u];
    }
  }
  __syncthreads();
  // rows are dealt exactly as in the pipelined path: 32-row blocks to warps
  // round-robin (continuing over the groups of an item), one row per lane
  constexpr int NW = kBlock / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (re - r + 31) >> 5;
  for (int j = (int)((uint32_t)(warp - (int)(blocks % NW) + NW) % NW); j < nblk; j += NW) {
    const int row = r + 32 * j + lane;
    if (row < re) {
      const int a0 = __ldg(rp + row) - base, a1 = __ldg(rp + row + 1) - base;
      const typename Op::Pre q = op.pre(row);
      AT sum = AT(0);
      for (int e = a0; e < a1; ++e) sum = rfma(Conv<AT>::f(ldro(val + base + e)), sbuf[e], sum);
      op.fin(row, sum, q, p0, p1);
    }
  }
  blocks += (uint32_t)nblk;
  __syncthreads();
}

// y_row = sum over the row's entries of val * op.gather(col), in stored
// order, then op.fin(row, y_row, op.pre(row)).  A tile whose entries fit the
// staging buffer is one group: each thread loads its rows' operands, issues
// all of its entry loads and gathers, stores the products in shared memory
// and sums its rows.  Larger tiles are split into groups by binary search;
// a row with more than kCap entries is summed by the whole block.
template <class AT, class MV, class Op>
__device__ __forceinline__ void spmv_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const MV* __restrict__ val, int r0, int r1, AT* sbuf, double* red,
                                          const Op& op, double& p0, double& p1, uint32_t& blocks) {
  const int t0 = __ldg(rp + r0), t1 = __ldg(rp + r1);
  if (t1 - t0 <= kCap) {
    spmv_group<AT>(rp, ci, val, r0, r1, t0, t1 - t0, sbuf, op, p0, p1, blocks);
    return;
  }
  int r = r0;
  while (r < r1) {
    const int base = __ldg(rp + r);
    int lo = r, hi = r1;
    while (lo < hi) {
      const int mid = lo + ((hi - lo + 1) >> 1);
      if (__ldg(rp + mid) - base <= kCap) lo = mid; else hi = mid - 1;
    }
    const int re = lo;
    if (re == r) {
      const int e1 = __ldg(rp + r + 1);
      double acc = 0.0;
      for (int e = base + threadIdx.x; e < e1; e += blockDim.x)
        acc = rfma((double)Conv<AT>::f(ldro(val + e)), (double)op.gather(__ldg(ci + e)), acc);
      acc = block_sum(acc, red);
      if (threadIdx.x == 0) {
        const typename Op::Pre pr = op.pre(r);
        op.fin(r, (AT)acc, pr, p0, p1);
      }
      __syncthreads();
      r += 1;
      continue;
    }
    spmv_group<AT>(rp, ci, val, r, re, base, __ldg(rp + re) - base, sbuf, op, p0, p1, blocks);
    r = re;
  }
}

// ---- per-phase operations: gather(col), pre(row) loads, fin(row, sum) ----
// W is the element stride of the four paired vectors.  W = 1: s, d, q and r
// are separate arrays.  W = 2: they are stored as interleaved pairs, s with d
// (s_i at 2i, d_i at 2i + 1 of the same buffer) and q with r, so the passes
// that gather two vectors at the same column (A: s and d; G^T: q and r) load
// both with one 8-byte (float) or 16-byte (double) access, one L2 sector
// request instead of two.  The arithmetic is the same for both strides.
template <class VT> struct Pair2;
template <> struct Pair2<float> { using T = float2; };
template <> struct Pair2<double> { using T = double2; };
template <class VT> __device__ __forceinline__ typename Pair2<VT>::T ldpair(const VT* p) {
  return *reinterpret_cast<const typename Pair2<VT>::T*>(p);
}

template <class VT, int W> struct OpP1 {   // p = s + beta d;  d' = p;  q = A p;  p.q
  const VT* s; const VT* dcur; VT* dnxt; VT* q; VT beta; bool first;   // W = 2: dcur = s + 1
  struct Pre { VT sv, dv; };
  __device__ VT gather(int c) const {
    if constexpr (W == 2) {
      const auto v = ldpair(s + 2 * (int64_t)c);
      return first ? v.x : rfma(beta, v.y, v.x);
    } else {
      const VT sv = ldv(s + c);
      return first ? sv : rfma(beta, ldv(dcur + c), sv);
    }
  }
  __device__ Pre pre(int row) const {
    if constexpr (W == 2) {
      const auto v = ldpair(s + 2 * (int64_t)row);
      return Pre{v.x, first ? VT(0) : v.y};
    } else {
      return Pre{ldv(s + row), first ? VT(0) : ldv(dcur + row)};
    }
  }
  __device__ void fin(int row, VT sum, const Pre& p, double& p0, double&) const {
    const VT pv = first ? p.sv : rfma(beta, p.dv, p.sv);
    dnxt[W * (int64_t)row] = pv;
    q[W * (int64_t)row] = sum;
    p0 += (double)pv * (double)sum;
  }
};
template <class VT, int W> struct OpP2 {   // x += alpha d;  r' = r - alpha q;  t = G^T r';  r'.r'
  const VT* rcur; VT* rnxt; const VT* q; const VT* dcur; VT* x; VT* t; VT alpha;   // W = 2: rcur = q + 1
  struct Pre { VT xv, dv, rv, qv; };
  __device__ VT gather(int c) const {
    if constexpr (W == 2) {
      const auto v = ldpair(q + 2 * (int64_t)c);
      return rfma(-alpha, v.x, v.y);
    } else {
      return rfma(-alpha, ldv(q + c), ldv(rcur + c));
    }
  }
  __device__ Pre pre(int row) const {
    if constexpr (W == 2) {
      const auto v = ldpair(q + 2 * (int64_t)row);
      return Pre{ldv(x + row), ldv(dcur + 2 * (int64_t)row), v.y, v.x};
    } else {
      return Pre{ldv(x + row), ldv(dcur + row), ldv(rcur + row), ldv(q + row)};
    }
  }
  __device__ void fin(int row, VT sum, const Pre& p, double& p0, double&) const {
    x[row] = rfma(alpha, p.dv, p.xv);
    const VT rn = rfma(-alpha, p.qv, p.rv);
    rnxt[W * (int64_t)row] = rn;
    t[row] = sum;
    p0 += (double)rn * (double)rn;
  }
};
template <class VT, int W> struct OpApply1 {   // t = G^T r
  const VT* r; VT* t;
  struct Pre {};
  __device__ VT gather(int c) const { return ldv(r + W * (int64_t)c); }
  __device__ Pre pre(int) const { return Pre{}; }
  __device__ void fin(int row, VT sum, const Pre&, double&, double&) const { t[row] = sum; }
};
template <class VT, int W> struct OpApply2 {   // s = G t + eps r;  r.s
  const VT* t; const VT* r; VT* s; VT eps;
  struct Pre { VT rv; };
  __device__ VT gather(int c) const { return ldv(t + c); }
  __device__ Pre pre(int row) const { return Pre{ldv(r + W * (int64_t)row)}; }
  __device__ void fin(int row, VT sum, const Pre& p, double& p0, double&) const {
    const VT sv = rfma(eps, p.rv, sum);
    s[W * (int64_t)row] = sv;
    p0 += (double)p.rv * (double)sv;
  }
};
template <class VT, int W> struct OpResid {   // r = b - A x;  r.r, b.b   (b float64)
  const VT* x; const double* b; VT* r;
  struct Pre { double bv; };
  __device__ VT gather(int c) const { return ldv(x + c); }
  __device__ Pre pre(int row) const { return Pre{__ldg(b + row)}; }
  __device__ void fin(int row, VT sum, const Pre& p, double& p0, double& p1) const {
    const VT rv = rsub((VT)p.bv, sum);
    r[W * (int64_t)row] = rv;
    p0 += (double)rv * (double)rv;
    p1 += p.bv * p.bv;
  }
};
template <class VT, int W> struct OpResidIn {   // r = rin - A e   (inner replacement, mixed)
  const VT* e; const VT* rin; VT* r;
  struct Pre { VT iv; };
  __device__ VT gather(int c) const { return ldv(e + c); }
  __device__ Pre pre(int row) const { return Pre{ldv(rin + row)}; }
  __device__ void fin(int row, VT sum, const Pre& p, double& p0, double&) const {
    const VT rv = rsub(p.iv, sum);
    r[W * (int64_t)row] = rv;
    p0 += (double)rv * (double)rv;
  }
};
template <class VT, int W> struct OpResid64 {   // r64 = b - A64 x64;  r = rin = (VT) r64;  e = 0
  const double* x64; const double* b; VT* r; VT* rin; VT* e;
  struct Pre { double bv; };
  __device__ double gather(int c) const { return ldv(x64 + c); }
  __device__ Pre pre(int row) const { return Pre{__ldg(b + row)}; }
  __device__ void fin(int row, double sum, const Pre& p, double& p0, double& p1) const {
    const double r64 = __dsub_rn(p.bv, sum);
    const VT r32 = (VT)r64;
    r[W * (int64_t)row] = r32;
    rin[row] = r32;
    e[row] = VT(0);
    p0 += r64 * r64;
    p1 += p.bv * p.bv;
  }
};

// ---- TMA-fed groups ----
// Shared memory of one block: kStages stages of (column indices, values) for
// one group each.  SELL-32 groups use every stage; CSR groups use one stage
// fewer in float32 kernels and keep the per-warp product buffers in the last
// one (float64 kernels: after the stages); the direct path's buffer overlays
// stage 0 (it runs only while the ring is idle: every piped call waits for
// all of the copies it issues).  Mbarriers and group headers are static.
template <class MV> struct StageLayout {
  static constexpr int kStageE = kCap + 2 * kAlignE;  // entries per stage buffer
  static constexpr int kColBytes = kStageE * 4;
  static constexpr int kValBytes = kStageE * (int)sizeof(MV);
  static constexpr int kStageBytes = kColBytes + kValBytes;
  static constexpr int kStages = sizeof(MV) == 4 ? kStagesSell32 : kStages64;  // stages in the region
  static constexpr int kCsrStages = sizeof(MV) == 4 ? kStages32 : kStages64;
};

struct GroupHdr {
  int r, re, e0, e0a, e1, r_al, staged, pad;
};

// The ring lives at fixed shared-memory addresses (no pointers held in
// registers): the stage region is the block's dynamic shared memory.
extern __shared__ __align__(128) unsigned char eng_smem[];
__shared__ uint64_t eng_bar[kStages];       // stage mbarriers
__shared__ GroupHdr eng_hdr[kStages];       // stage group headers
__shared__ int eng_grow[kMaxK + 1];         // group row (or slice) starts of the current item
__shared__ int eng_gent[kMaxK + 1];         // group first entries
__shared__ int eng_rel[kStages];            // warps done with the stage's group

// Per-thread ring state (uniform over the block).
struct Pipe {
  uint32_t par;  // parity of the next phase of each stage mbarrier
  bool ok;       // false once a stage wait of this thread timed out
};

// Waits for stage st; false (and the error flag set) if it did not arrive in
// time or an earlier wait of this warp timed out, so that a stage that may
// hold stale column indices is never gathered from.
__device__ __forceinline__ bool stage_wait(Pipe& P, int st, uint64_t limit_ns, int* err) {
  if (!mbar_wait_bounded(eng_bar + st, (P.par >> st) & 1u, limit_ns)) {
    atomicExch(err, SPAI_ERR_TIMEOUT);
    P.ok = false;
  }
  P.par ^= 1u << st;
  return __all_sync(0xffffffffu, P.ok);
}

template <class AT> __device__ __forceinline__ unsigned char* stage_ptr(int st) {
  return eng_smem + (size_t)st * StageLayout<AT>::kStageBytes;
}

// Thread 0: bulk-copy the entries of group g (rows tiles[g]..tiles[g+1]) into
// the next stage.  Copies start at a multiple of kAlignE entries (16-byte
// aligned for every value type) and the arrays are padded past nnz.
template <class AT, class MV>
__device__ __forceinline__ void issue_group(const int32_t* ci, const MV* val, int k, int st) {
  const int r = eng_grow[k], re = eng_grow[k + 1];
  const int e0 = eng_gent[k], e1 = eng_gent[k + 1];
  const int e0a = e0 & ~(kAlignE - 1);
  int ne = ((e1 + kAlignE - 1) & ~(kAlignE - 1)) - e0a;
  if (ne < kAlignE) ne = kAlignE;
  eng_hdr[st] = GroupHdr{r, re, e0, e0a, e1, 0, 0, 0};
  unsigned char* base = stage_ptr<AT>(st);
  const unsigned cb = (unsigned)ne * 4u, vb = (unsigned)ne * (unsigned)sizeof(MV);
  mbar_arrive_expect_tx(eng_bar + st, cb + vb);
  const uint64_t pol = l2_evict_first_policy();
  tma_load_1d_hint(base, ci + e0a, cb, eng_bar + st, pol);
  tma_load_1d_hint(base + StageLayout<AT>::kColBytes, val + e0a, vb, eng_bar + st, pol);
}

// Processes groups [g0, g1) of one matrix through the stage ring.  Warps work
// independently: each takes 32-row blocks of every staged group (blocks are
// dealt round-robin over the warps, continuing across groups), one row per
// lane for the sums and all 32 lanes for the entry gathers, with a private
// product buffer and only warp-level synchronisation.  A stage is released
// when every warp is done with its group; the warp that releases it last
// issues the bulk copy of the group kStages further on into it.
template <int NS, class AT, class MV, class Op>
__device__ __forceinline__ void piped_groups(Pipe& P, const int32_t* __restrict__ tiles,
                                             const int32_t* __restrict__ rp, const int32_t* ci, const MV* val,
                                             int g0, int g1, const Op& op, double& p0, double& p1,
                                             uint64_t limit_ns, int* err) {
  const int ng = g1 - g0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kBlock / 32;
  // bounds of every group of this item (row start, first entry), loaded once
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) {
    const int r = __ldg(tiles + g0 + i);
    eng_grow[i] = r;
    eng_gent[i] = __ldg(rp + r);
  }
  if (threadIdx.x < NS) eng_rel[threadIdx.x] = 0;
  fence_async_smem();  // earlier generic writes to the stages precede the bulk copies
  __syncthreads();
  if (threadIdx.x == 0) {
    const int pre = ng < NS ? ng : NS;
    for (int k = 0; k < pre; ++k) issue_group<AT, MV>(ci, val, k, k);
  }
  AT* wb = reinterpret_cast<AT*>(stage_ptr<AT>(StageLayout<AT>::kCsrStages)) + warp * kWarpE;
  uint32_t blocks = 0;  // the deal of row blocks to warps restarts with every item
  for (int k = 0; k < ng; ++k) {
    const int st = k % NS;
    const bool go = stage_wait(P, st, limit_ns, err);
    const GroupHdr h = eng_hdr[st];
    const unsigned char* base = stage_ptr<AT>(st);
    const int32_t* cs = reinterpret_cast<const int32_t*>(base) - h.e0a;  // indexed by entry offset
    const MV* vs = reinterpret_cast<const MV*>(base + StageLayout<AT>::kColBytes) - h.e0a;
    const int nrows = h.re - h.r;
    const int nblk = (nrows + 31) >> 5;
    // first block of this group owned by this warp
    int j = (int)((uint32_t)(warp - (int)(blocks % NW) + NW) % NW);
    for (; go && j < nblk; j += NW) {
      const int row = h.r + 32 * j + lane;
      const bool valid = row < h.re;
      int ea = 0, eb = 0;
      typename Op::Pre pr;
      if (valid) {
        ea = __ldg(rp + row);
        eb = __ldg(rp + row + 1);
        pr = op.pre(row);
      }
      const int last = min(31, h.re - (h.r + 32 * j) - 1);
      const int E0 = __shfl_sync(0xffffffffu, ea, 0);
      const int E1 = __shfl_sync(0xffffffffu, eb, last);
      AT acc = AT(0);
      for (int cb = E0; cb < E1; cb += kWarpE) {
        const int m = min(kWarpE, E1 - cb);
        int cix[kWarpE / 32];
#pragma unroll
        for (int u = 0; u < kWarpE / 32; ++u) {
          const int kk = lane + 32 * u;
          cix[u] = (kk < m) ? cs[cb + kk] : 0;
        }
        AT g[kWarpE / 32];
#pragma unroll
        for (int u = 0; u < kWarpE / 32; ++u) {
          const int kk = lane + 32 * u;
          g[u] = (kk < m) ? op.gather(cix[u]) : AT(0);
        }
#pragma unroll
        for (int u = 0; u < kWarpE / 32; ++u) {
          const int kk = lane + 32 * u;
          if (kk < m) wb[kk] = g[u];
        }
        __syncwarp();
        if (valid) {
          const int lo = max(ea, cb), hi = min(eb, cb + m);
          for (int e = lo; e < hi; ++e) acc = rfma(Conv<AT>::f(vs[e]), wb[e - cb], acc);
        }
        __syncwarp();
      }
      if (valid) op.fin(row, acc, pr, p0, p1);
    }
    blocks += (uint32_t)nblk;
    // release the stage; the last warp refills it
    if (lane == 0) {
      __threadfence_block();
      const int prev = atomicAdd(eng_rel + st, 1);
      if (prev == NW - 1) {
        eng_rel[st] = 0;
        if (k + NS < ng) issue_group<AT, MV>(ci, val, k + NS, st);
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// SELL-32 groups [g0, g1) (a group = consecutive 32-row slices) through the
// same stage ring: each slice is taken by one warp (slices dealt round-robin
// over the warps, continuing across groups), lane l owns row 32 s + l, loads
// its entries column-major from the staged slice (conflict-free), issues all
// gathers of a batch of 8 entries before summing them, and sums its row in
// stored order -- the same per-row arithmetic as the CSR path, without the
// product buffer.
template <int NS, class AT, class MV, class Op>
__device__ __forceinline__ void piped_slices(Pipe& P, const int32_t* __restrict__ tiles,
                                             const int32_t* __restrict__ sptr, const int32_t* __restrict__ rp,
                                             const int32_t* ci, const MV* val, int g0, int g1, int64_t n,
                                             const Op& op, double& p0, double& p1, uint64_t limit_ns, int* err,
                                             const int32_t* __restrict__ srow) {
  const int ng = g1 - g0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kBlock / 32;
  constexpr int kB = 8;
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) {
    const int sl = __ldg(tiles + g0 + i);
    eng_grow[i] = sl;
    eng_gent[i] = __ldg(sptr + sl);
  }
  if (threadIdx.x < NS) eng_rel[threadIdx.x] = 0;
  fence_async_smem();  // earlier generic writes to the stages precede the bulk copies
  __syncthreads();
  if (threadIdx.x == 0) {
    const int pre = ng < NS ? ng : NS;
    for (int k = 0; k < pre; ++k) issue_group<AT, MV>(ci, val, k, k);
  }
  uint32_t blocks = 0;
  for (int k = 0; k < ng; ++k) {
    const int st = k % NS;
    // slice offsets of the group, loaded before the wait (the group's slice
    // range is known from the item): lane l holds sptr[first + l] and
    // sptr[first + 32 + l]
    const int gs0 = eng_grow[k];
    const int nsl = eng_grow[k + 1] - gs0;
    const int so0 = lane <= nsl ? __ldg(sptr + gs0 + lane) : 0;
    const int so1 = lane + 32 <= nsl ? __ldg(sptr + gs0 + 32 + lane) : 0;
    const bool go = stage_wait(P, st, limit_ns, err);
    const GroupHdr h = eng_hdr[st];
    const unsigned char* base = stage_ptr<AT>(st);
    const int32_t* cs = reinterpret_cast<const int32_t*>(base) - h.e0a;
    const MV* vs = reinterpret_cast<const MV*>(base + StageLayout<AT>::kColBytes) - h.e0a;
    int j = (int)((uint32_t)(warp - (int)(blocks % NW) + NW) % NW);
    for (; go && j < nsl; j += NW) {
      const int sl = gs0 + j;
      int off, end;
      if (nsl <= kSlicesInReg) {
        off = __shfl_sync(0xffffffffu, j < 32 ? so0 : so1, j & 31);
        end = __shfl_sync(0xffffffffu, j + 1 < 32 ? so0 : so1, (j + 1) & 31);
      } else {
        off = __ldg(sptr + sl);
        end = __ldg(sptr + sl + 1);
      }
      const int w = (end - off) >> 5;
      const int row = srow ? __ldg(srow + (size_t)sl * 32 + lane) : sl * 32 + lane;
      const bool valid = row < n;
      typename Op::Pre pr;
      if (valid) pr = op.pre(row);
      // padding entries (beyond a row's length) hold column 0 and value 0:
      // they add exact zeros, so no row lengths are needed
      const int32_t* cl = cs + off + lane;
      const MV* vl = vs + off + lane;
      AT acc = AT(0);
      for (int k0 = 0; k0 < w; k0 += kB) {
        AT gv[kB];  // all gathers of the batch in flight before the sums
#pragma unroll
        for (int u = 0; u < kB; ++u) gv[u] = (k0 + u < w) ? op.gather(cl[32 * (k0 + u)]) : AT(0);
#pragma unroll
        for (int u = 0; u < kB; ++u)
          if (k0 + u < w) acc = rfma(Conv<AT>::f(vl[32 * (k0 + u)]), gv[u], acc);
      }
      if (valid) op.fin(row, acc, pr, p0, p1);
    }
    blocks += (uint32_t)nsl;
    if (lane == 0) {
      __threadfence_block();
      const int prev = atomicAdd(eng_rel + st, 1);
      if (prev == NW - 1) {
        eng_rel[st] = 0;
        if (k + NS < ng) issue_group<AT, MV>(ci, val, k + NS, st);
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Groups [g0, g1) without the stage ring (rows longer than a group, or the
// float64 residual of mixed precision): direct loads.  Not inlined (rarely
// run), so everything crosses the call by value: the item's partial sums
// come back as the result instead of through references, which would keep
// the caller's accumulators in local memory.
template <class AT, class MV, class Op>
__device__ __noinline__ double2 direct_groups(const int32_t* __restrict__ tiles, const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ ci, const MV* __restrict__ val, int g0,
                                              int g1, AT* sbuf, double* red, const Op op) {
  uint32_t blocks = 0;
  double p0 = 0.0, p1 = 0.0;
  for (int g = g0; g < g1; ++g)
    spmv_rows<AT>(rp, ci, val, __ldg(tiles + g), __ldg(tiles + g + 1), sbuf, red, op, p0, p1, blocks);
  return make_double2(p0, p1);
}

// Rows [r0, r1) without the stage ring (float64 residual of mixed precision
// over SELL-32 slices): direct loads.
template <class AT, class MV, class Op>
__device__ __noinline__ double2 direct_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                            const MV* __restrict__ val, int r0, int r1, AT* sbuf, double* red,
                                            const Op op) {
  uint32_t blocks = 0;
  double p0 = 0.0, p1 = 0.0;
  spmv_rows<AT>(rp, ci, val, r0, r1, sbuf, red, op, p0, p1, blocks);
  return make_double2(p0, p1);
}

// Rows covered by one tile unit of a format: a CSR row, a 32-row slice, or a
// slice of 32 block rows (96 scalar rows).
__host__ __device__ __forceinline__ int rows_per_unit(int fmt) { return fmt == 1 ? 32 : (fmt == 2 ? 96 : 1); }

// Slices [tiles[g0], tiles[g1]) of the 3 x 3 block layout (bsell.cu), direct
// loads: a warp per slice (slices dealt to warps round-robin), a lane per
// block row I (scalar rows 3I .. 3I + 2).  Per block: its column J, the three
// gathers at 3J .. 3J + 2 and its 9 values; each scalar row sums its entries
// in stored order (blocks in column order, columns within a block in order),
// the per-row arithmetic of the scalar layouts.  Two blocks are in flight per
// step.  Not inlined (its registers stay out of the scalar paths).
template <class AT, class MV, class Op>
__device__ __noinline__ double2 direct_bslices(const int32_t* __restrict__ tiles, const int32_t* __restrict__ sptr,
                                               const int32_t* __restrict__ ci, const MV* __restrict__ val, int g0,
                                               int g1, int64_t n, const Op op) {
  constexpr int NW = kBlock / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double p0 = 0.0, p1 = 0.0;
  const int s0 = __ldg(tiles + g0), s1 = __ldg(tiles + g1);
  for (int sl = s0 + warp; sl < s1; sl += NW) {
    const int off = __ldg(sptr + sl);
    const int w = (__ldg(sptr + sl + 1) - off) >> 5;
    const int64_t row0 = 3 * ((int64_t)sl * 32 + lane);
    const bool valid = row0 < n;
    typename Op::Pre pr[3];
    if (valid) {
#pragma unroll
      for (int r = 0; r < 3; ++r) pr[r] = op.pre((int)row0 + r);
    }
    AT acc[3] = {AT(0), AT(0), AT(0)};
    const int32_t* cl = ci + off + lane;
    const MV* vl = val + 9 * (size_t)off + lane;
    for (int q = 0; q < w; q += 2) {
      const bool two = q + 1 < w;
      const int j0 = __ldg(cl + 32 * q);
      const int j1 = two ? __ldg(cl + 32 * (q + 1)) : 0;
      AT v0[9], v1[9], x0[3], x1[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        v0[k] = Conv<AT>::f(ldro(vl + 32 * (9 * q + k)));
        v1[k] = two ? Conv<AT>::f(ldro(vl + 32 * (9 * (q + 1) + k))) : AT(0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x0[c] = op.gather(3 * j0 + c);
        x1[c] = two ? op.gather(3 * j1 + c) : AT(0);
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r] = rfma(v0[3 * r + c], x0[c], acc[r]);
        if (two) {
#pragma unroll
          for (int c = 0; c < 3; ++c) acc[r] = rfma(v1[3 * r + c], x1[c], acc[r]);
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int r = 0; r < 3; ++r) op.fin((int)row0 + r, acc[r], pr[r], p0, p1);
    }
  }
  return make_double2(p0, p1);
}

// CSR: the kernel streams CSR groups through the ring; kernels for launches
// without such groups (every member SELL-32 or direct) leave that code out,
// which keeps the SELL-32 loop free of its register pressure.
template <class AT, bool CSR, class MV, class Op>
__device__ __forceinline__ void run_groups(bool piped, Pipe& P, const int32_t* tiles, const int32_t* rp,
                                           const int32_t* ci, const MV* val, int g0, int g1, void* sbuf,
                                           double* red, const Op& op, double& p0, double& p1, uint64_t limit_ns,
                                           int* err, const int32_t* sptr, int64_t n, const int32_t* srow) {
  if (sptr) piped_slices<(sizeof(AT) == 4 ? kStagesSell32 : kStages64), AT, MV>(P, tiles, sptr, rp, ci, val, g0, g1, n,
                                                                          op, p0, p1, limit_ns, err, srow);
  else if (CSR && piped) {
    if constexpr (CSR)
      piped_groups<(sizeof(AT) == 4 ? kStages32 : kStages64), AT, MV>(P, tiles, rp, ci, val, g0, g1, op, p0, p1,
                                                                     limit_ns, err);
  } else {
    const double2 q = direct_groups<AT, MV>(tiles, rp, ci, val, g0, g1, reinterpret_cast<AT*>(sbuf), red, op);
    p0 += q.x;
    p1 += q.y;
  }
}

// Kernel variants: KV 0 streams SELL-32 slices in row order only, KV 1 also
// row-mapped slices (rows sorted by length), KV 2 everything (CSR row groups
// through the ring, the 3 x 3 block layout, row maps).  A launch runs the
// smallest variant its members need: each extra path costs the SELL-32 loop
// registers and time.
// W = 2 (paired vectors) only in variants 1 and 2.
template <class VT, class GT, bool MIXED, int KV, int W>
__device__ void run_item_w(int ph, const EngSys& S, const EngState& st, int g0, int g1, Pipe& P, void* sbuf,
                           double* red, double& p0, double& p1, uint64_t limit_ns, int* err, int rc) {
  constexpr bool CSR = KV == 2;
  const int dc = st.dc;
  VT* r_cur = reinterpret_cast<VT*>(S.r[rc]);
  VT* r_nxt = reinterpret_cast<VT*>(S.r[rc ^ 1]);
  VT* d_cur = reinterpret_cast<VT*>(S.d[dc]);
  VT* d_nxt = reinterpret_cast<VT*>(S.d[dc ^ 1]);
  // paired: q shares r[rc]'s buffer (q_i at 2i, r_i at 2i + 1), s shares d[dc]'s
  VT* q_v = W == 2 ? r_cur - 1 : reinterpret_cast<VT*>(S.q);
  VT* t = reinterpret_cast<VT*>(S.t);
  VT* s = W == 2 ? d_cur - 1 : reinterpret_cast<VT*>(S.s);
  VT* xv = MIXED ? reinterpret_cast<VT*>(S.e) : reinterpret_cast<VT*>(S.x);  // iterate
  VT* rin = reinterpret_cast<VT*>(S.rin);
  const VT* aval = reinterpret_cast<const VT*>(S.val[MAT_A]);
  const GT* gtval = reinterpret_cast<const GT*>(S.val[MAT_GT]);
  const GT* gval = reinterpret_cast<const GT*>(S.val[MAT_G]);
  const VT alpha = (VT)st.alpha, beta = (VT)st.beta, eps = (VT)S.eps;
  const int m = phase_mat(ph);
  const int32_t* tl = S.tiles[m];
  const bool piped = S.fits[m] != 0;
  const int32_t* sp = S.fmt[m] == 1 ? S.sptr[m] : nullptr;  // SELL-32 slices
  // their rows when sorted by length: a row map only variants 1 and 2 read,
  // so the plain SELL-32 kernel's loop stays as it was
  const int32_t* srow = (KV >= 1 && S.fmt[m] == 1) ? S.srow[m] : nullptr;
  const int64_t n = S.n;
  const int rpu = rows_per_unit(S.fmt[m]);
  // 3 x 3 block layout: compiled into the full kernel only (launches with a
  // block member run it), so the SELL-32 kernel keeps its registers
  if (CSR && S.fmt[m] == 2 && ph != PH_RESID64 && ph != PH_P2X && ph != PH_XUPD && ph != PH_ZEROX) {
    double2 q = make_double2(0.0, 0.0);
    if constexpr (CSR) switch (ph) {
      case PH_P1:
        q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_A], aval, g0, g1, n,
                               OpP1<VT, W>{s, d_cur, d_nxt, q_v, beta, st.first != 0});
        break;
      case PH_P2:
        q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_GT], gtval, g0, g1, n,
                               OpP2<VT, W>{r_cur, r_nxt, q_v, d_cur, xv, t, alpha});
        break;
      case PH_APPLY1:
        q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_GT], gtval, g0, g1, n, OpApply1<VT, W>{r_cur, t});
        break;
      case PH_APPLY2:
        q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_G], gval, g0, g1, n, OpApply2<VT, W>{t, r_cur, s, eps});
        break;
      case PH_RESID0:
      case PH_RESID:
        if (!MIXED) q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_A], aval, g0, g1, n, OpResid<VT, W>{xv, S.b, r_cur});
        else q = direct_bslices<VT>(tl, S.sptr[m], S.ci[MAT_A], aval, g0, g1, n, OpResidIn<VT, W>{xv, rin, r_cur});
        break;
      default:
        break;
    }
    p0 += q.x;
    p1 += q.y;
    return;
  }

  switch (ph) {
    case PH_P1: {
      OpP1<VT, W> op{s, d_cur, d_nxt, q_v, beta, st.first != 0};
      run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_A], S.ci[MAT_A], aval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      break;
    }
    case PH_P2: {
      OpP2<VT, W> op{r_cur, r_nxt, q_v, d_cur, xv, t, alpha};
      run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_GT], S.ci[MAT_GT], gtval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      break;
    }
    case PH_APPLY1: {
      OpApply1<VT, W> op{r_cur, t};
      run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_GT], S.ci[MAT_GT], gtval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      break;
    }
    case PH_APPLY2: {
      OpApply2<VT, W> op{t, r_cur, s, eps};
      run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_G], S.ci[MAT_G], gval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      break;
    }
    case PH_RESID0:
    case PH_RESID: {
      if (!MIXED) {
        OpResid<VT, W> op{xv, S.b, r_cur};
        run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_A], S.ci[MAT_A], aval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      } else {
        OpResidIn<VT, W> op{xv, rin, r_cur};
        run_groups<VT, CSR>(piped, P, tl, S.rp[MAT_A], S.ci[MAT_A], aval, g0, g1, sbuf, red, op, p0, p1, limit_ns, err, sp, n, srow);
      }
      break;
    }
    case PH_RESID64: {
      if constexpr (MIXED) {
        OpResid64<VT, W> op{S.x, S.b, r_cur, rin, xv};
        if (rpu > 1) {  // the rows of slices [tl[g0], tl[g1]) over the CSR copy of A
          const int r0 = __ldg(tl + g0) * rpu, r1 = (int)min((int64_t)__ldg(tl + g1) * rpu, n);
          if (r0 < r1) {
            const double2 q =
                direct_rows<double>(S.rp[MAT_A], S.a_ci64, S.a_v64, r0, r1, reinterpret_cast<double*>(sbuf), red, op);
            p0 += q.x;
            p1 += q.y;
          }
        } else {
          const double2 q =
              direct_groups<double>(tl, S.rp[MAT_A], S.a_ci64, S.a_v64, g0, g1, reinterpret_cast<double*>(sbuf), red, op);
          p0 += q.x;
          p1 += q.y;
        }
      }
      break;
    }
    case PH_P2X:
    case PH_XUPD:
    case PH_ZEROX: {
      const int r0 = __ldg(tl + g0) * rpu;
      const int r1 = (int)min((int64_t)__ldg(tl + g1) * rpu, n);
      for (int row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
        if (ph == PH_P2X) xv[row] = rfma(alpha, ldv(d_cur + W * (int64_t)row), ldv(xv + row));
        else if (ph == PH_XUPD) {
          S.x[row] = __dadd_rn(ldv(S.x + row), (double)ldv(xv + row));
          xv[row] = VT(0);
        }
        else S.x[row] = 0.0;
      }
      break;
    }
    default:
      break;
  }
}

// The paired path is a separate function so that the kernel's own loop keeps
// the registers of the separate-vector path (one call per work item).
template <class VT, class GT, bool MIXED, int KV>
__device__ __noinline__ void run_item_pair(int ph, const EngSys& S, const EngState& st, int g0, int g1, Pipe& P,
                                           void* sbuf, double* red, double* pp, uint64_t limit_ns, int* err, int rc) {
  double p0 = pp[0], p1 = pp[1];
  run_item_w<VT, GT, MIXED, KV, 2>(ph, S, st, g0, g1, P, sbuf, red, p0, p1, limit_ns, err, rc);
  pp[0] = p0;
  pp[1] = p1;
}

template <class VT, class GT, bool MIXED, int KV>
__device__ __forceinline__ void run_item(int ph, const EngSys& S, const EngState& st, int g0, int g1, Pipe& P,
                                         void* sbuf, double* red, double& p0, double& p1, uint64_t limit_ns, int* err,
                                         int rc) {
  if constexpr (KV >= 1) {
    if (S.pair) {
      double pp[2] = {p0, p1};
      run_item_pair<VT, GT, MIXED, KV>(ph, S, st, g0, g1, P, sbuf, red, pp, limit_ns, err, rc);
      p0 = pp[0];
      p1 = pp[1];
      return;
    }
  }
  run_item_w<VT, GT, MIXED, KV, 1>(ph, S, st, g0, g1, P, sbuf, red, p0, p1, limit_ns, err, rc);
}

// State machine of one system; runs once per phase in the block that
// completes the system's last work item.  float64 mode follows Algorithm 1
// with the reading documented in the oracle: the true residual replaces r on
// iterations i % period == 0 and confirms convergence.  Mixed mode keeps the
// same iteration in float32 and replaces r by the float64 true residual
// b - A x (after folding the float32 correction e into the float64 x):
// every `period` iterations, when ||r|| has dropped by `reliable` since the
// last replacement, and to confirm convergence.  The Krylov recurrence is not
// restarted (beta continues from delta_old), so float64 accuracy is reached
// in about the float64 iteration count.
template <bool MIXED>
__device__ void transition(const EngSys& S, EngState& st, double q0, double q1, const EngOpts& o, GridSync* gs) {
  auto finish = [&](int status) {
    st.status = status;
    st.phase = PH_DONE;
    atomicSub(&gs->live, 1);
  };
  auto hist = [&](double v) {
    if (S.history && st.hist_n < S.history_len) S.history[st.hist_n] = v;
    st.hist_n++;
  };
  const int RESID_PH = MIXED ? PH_XUPD : PH_RESID;  // how a true residual is obtained
  switch (st.phase) {
    case PH_RESID0:
    case PH_RESID64:
    case PH_RESID: {
      const bool initial = (st.phase == PH_RESID0) || (MIXED && st.first_resid == 0);
      st.rr = q0;
      if (initial) {
        st.bb = q1;
        st.first_resid = 1;
        hist(sqrt(q0));
        if (st.bb == 0.0) { st.phase = PH_ZEROX; return; }
        if (o.criterion == SPAI_CRIT_RESIDUAL && st.rr <= o.tol2 * st.bb) { finish(SPAI_OK); return; }
        st.rr_ref = st.rr;
        st.first = 1;
        st.phase = PH_APPLY1;
        return;
      }
      if (MIXED) st.outer++;
      hist(sqrt(st.rr));
      st.rr_ref = st.rr;
      if (o.criterion == SPAI_CRIT_RESIDUAL && st.rr <= o.tol2 * st.bb) { finish(SPAI_OK); return; }
      if (st.iter >= o.max_iter || st.stop) { finish(SPAI_ERR_NOT_CONVERGED); return; }
      if (MIXED && o.max_outer > 0 && st.outer >= o.max_outer) { finish(SPAI_ERR_NOT_CONVERGED); return; }
      st.phase = PH_APPLY1;
      return;
    }
    case PH_ZEROX:
      st.rr = 0.0;
      finish(SPAI_OK);
      return;
    case PH_APPLY1:
      st.phase = PH_APPLY2;
      return;
    case PH_APPLY2: {
      const double dn = q0;
      if (!(dn > 0.0) || !isfinite(dn)) {
        finish((o.criterion == SPAI_CRIT_PRECOND && dn == 0.0) ? SPAI_OK : SPAI_ERR_BREAKDOWN);
        return;
      }
      if (st.first) {
        st.delta0 = dn;
      } else {
        st.beta = dn / st.delta;
        if (S.lanczos && st.iter >= 1 && st.iter <= S.lanczos_len) S.lanczos[2 * (st.iter - 1) + 1] = st.beta;
      }
      st.delta = dn;
      if (o.criterion == SPAI_CRIT_PRECOND && !(dn > o.tol2 * st.delta0)) {
        if (MIXED && st.e_dirty) { st.stop_ok = 1; st.phase = PH_XUPD; return; }
        finish(SPAI_OK);
        return;
      }
      st.phase = PH_P1;
      return;
    }
    case PH_P1: {
      const double dq = q0;
      st.first = 0;
      st.dc ^= 1;
      if (!(dq > 0.0) || !isfinite(dq)) { finish(SPAI_ERR_BREAKDOWN); return; }
      st.alpha = st.delta / dq;
      if (S.lanczos && st.iter < S.lanczos_len) S.lanczos[2 * st.iter] = st.alpha;
      st.phase = (o.period > 0 && (st.iter % o.period) == 0) ? PH_P2X : (S.fuse ? PH_P2F : PH_P2);
      return;
    }
    case PH_P2: {
      st.rc ^= 1;
      st.iter++;
      st.e_dirty = 1;
      st.rr = q0;
      if (o.criterion == SPAI_CRIT_RESIDUAL && st.rr <= o.tol2 * st.bb) {
        st.phase = RESID_PH;  // confirm with the true residual
        return;
      }
      if (MIXED && st.rr <= o.reliable2 * st.rr_ref) {
        st.phase = PH_XUPD;  // reliable update
        return;
      }
      hist(sqrt(st.rr));
      if (st.iter >= o.max_iter) {
        if (MIXED) { st.stop = 1; st.phase = PH_XUPD; return; }
        finish(SPAI_ERR_NOT_CONVERGED);
        return;
      }
      st.phase = PH_APPLY2;
      return;
    }
    case PH_P2X:
      st.iter++;
      st.e_dirty = 1;
      st.phase = RESID_PH;
      return;
    case PH_XUPD:
      st.e_dirty = 0;
      if (st.stop_ok) { finish(SPAI_OK); return; }
      st.phase = PH_RESID64;
      return;
    default:
      return;
  }
}

// The state of one system into shared memory: one 8-byte word per lane of
// the first half-warp, so the 128-byte line arrives in one warp-wide request
// (every block reads the same line right after the grid barrier).
__device__ __forceinline__ void load_state(const EngState* src, EngState* dst) {
  constexpr int kWords = (int)(sizeof(EngState) / 8);
  static_assert(kWords <= 32, "one word per lane");
  if (threadIdx.x < kWords)
    reinterpret_cast<unsigned long long*>(dst)[threadIdx.x] =
        __ldcg(reinterpret_cast<const unsigned long long*>(src) + threadIdx.x);
}

template <class VT, class GT, bool MIXED, int KV>
__global__ void __launch_bounds__(kBlock, 3) engine_kernel(EngArgs a) {
  using MVmax = typename std::conditional<MIXED, float, double>::type;
  __shared__ double red[64];
  __shared__ int sflag, s_last, s_sys;
  __shared__ EngState s_st;

  Pipe P;
  P.par = 0;
  P.ok = true;
  void* sbuf = eng_smem;  // overlays stage 0: the ring is idle whenever the direct path runs
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(eng_bar + i, 1);  // every ring depth uses a prefix
    fence_mbar_init();
  }
  __syncthreads();

  const int slot0 = *(volatile int*)&a.gs->slot;
  const int npos = *(volatile int*)&a.gs->npos;  // fixed for the launch (re-dealt only between launches)
  bool skipped = false;  // the last item left without its closing block barrier
  int slots = 0;
  for (;;) {
    const int par = (slot0 + slots) & 1;
    EngState* cur = par ? a.st1 : a.st0;
    EngState* nxt = par ? a.st0 : a.st1;
    const unsigned epoch = (unsigned)(slot0 + slots) + 1u;
    // Pass 0 runs every system's phase; pass 1 only the G pass of fused
    // steps (PH_P2F), whose items wait for the flags pass 0 published.  The
    // item at table position p runs in block p % grid in both passes; a
    // block finishes its pass-0 items before it waits in pass 1.
    // `cur` changes within a slot only by finished systems, so the items of
    // fused steps are the same in both passes: a block that met none in
    // pass 0 has nothing to do in pass 1
    bool any_fused = false;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && !any_fused) break;
      int cached = -1;
      for (int it = blockIdx.x; it < npos; it += gridDim.x) {
        const int sid = __ldg(a.item_sys + it);
        if (sid < 0) continue;  // a hole of the last round
        const int v = __ldg(a.item_tile + it);
        if (sid >= a.nsys) {  // a corrupt table entry: flag it, skip it
          if (threadIdx.x == 0) atomicCAS(&a.gs->err, 0, kErrTable);
          continue;
        }
        if (sid != cached) {
          // a skipped item below leaves without the closing barrier: wait
          // until every warp has read the state it replaces
          if (skipped) __syncthreads();
          load_state(cur + sid, &s_st);
          __syncthreads();
          cached = sid;
          skipped = false;
        }
        const int ph0 = s_st.phase;
        if (ph0 == PH_DONE) {
          skipped = true;
          continue;
        }
        const bool fused = ph0 == PH_P2F;
        any_fused |= fused;
        if (pass == 1 && !fused) {
          skipped = true;
          continue;
        }
        const int ph = fused ? (pass == 0 ? PH_P2 : PH_APPLY2) : ph0;
        const EngSys& S = a.sys[sid];
        const int m = phase_mat(ph);
        const int K = S.kgroups[m];
        if (v < 0 || v >= S.nitems) {  // a corrupt table entry: flag it, skip it
          if (threadIdx.x == 0) atomicCAS(&a.gs->err, 0, kErrTable);
          skipped = true;
          continue;
        }
        const int g0 = v * K;
        int g1 = g0 + K;
        if (g1 > S.ntiles[m]) g1 = S.ntiles[m];
        if (pass == 1)  // the G^T items whose rows this item's G rows reach are done
          wait_items(ItemWait{a.flags + S.item_base, __ldg(S.dep + 2 * v), __ldg(S.dep + 2 * v + 1), epoch},
                     a.limit_ns, &a.gs->err);
        // the G pass of a fused step reads r' = r - alpha q, which the G^T pass wrote to r[rc ^ 1]
        const int rc = pass == 1 ? (s_st.rc ^ 1) : s_st.rc;
        double p0 = 0.0, p1 = 0.0;
        if (g0 < g1) run_item<VT, GT, MIXED, KV>(ph, S, s_st, g0, g1, P, sbuf, red, p0, p1, a.limit_ns, &a.gs->err,
                                                  rc);
        block_sum2(p0, p1, red);
        double* pbase = a.partial + 2 * (size_t)S.item_base;
        if (fused && pass == 0) {
          // the G^T pass of a fused step: keep r'.r' for the step's reduction, publish the item
          if (threadIdx.x == 0) {
            pbase[2 * v + 1] = p0;
            st_release_u32(a.flags + S.item_base + v, epoch);
          }
          continue;
        }
        double* cbase = a.cpartial + 2 * (size_t)S.chunk_base;
        const int nit = S.nitems;
        const int nch = (nit + kChunk - 1) / kChunk;
        const int ch = v / kChunk;
        const int ch_size = min(kChunk, nit - ch * kChunk);
        if (threadIdx.x == 0) {
          pbase[2 * v] = p0;
          if (!fused) pbase[2 * v + 1] = p1;
          const unsigned prev = atom_add_acq_rel_u32(a.ccnt + S.chunk_base + ch, 1u);
          s_last = (prev == (unsigned)(ch_size - 1)) ? 1 : 0;
        }
        __syncthreads();
        // s_last is read by every thread here and written again only after
        // the next item's reduction barriers; the system decision goes to
        // s_sys, so no warp can see it change before it has read it
        if (s_last) {
          // this block completed chunk `ch`: sum its item partials (one warp, fixed tree)
          if (threadIdx.x < 32) {
            const int tt = ch * kChunk + threadIdx.x;
            double c0 = (threadIdx.x < ch_size) ? __ldcg(pbase + 2 * tt) : 0.0;
            double c1 = (threadIdx.x < ch_size) ? __ldcg(pbase + 2 * tt + 1) : 0.0;
            c0 = warp_sum(c0);
            c1 = warp_sum(c1);
            if (threadIdx.x == 0) {
              cbase[2 * ch] = c0;
              cbase[2 * ch + 1] = c1;
              a.ccnt[S.chunk_base + ch] = 0u;
              const unsigned prev = atom_add_acq_rel_u32(a.cnt + sid, 1u);
              s_sys = (prev == (unsigned)(nch - 1)) ? 1 : 0;
            }
          }
          __syncthreads();
          if (s_sys) {
            double q0 = 0.0, q1 = 0.0;
            for (int tt = threadIdx.x; tt < nch; tt += blockDim.x) {
              q0 += __ldcg(cbase + 2 * tt);
              q1 += __ldcg(cbase + 2 * tt + 1);
            }
            block_sum2(q0, q1, red);
            if (threadIdx.x == 0) {
              EngState ns = s_st;
              if (fused) {
                // G^T pass (r'.r' in q1), then, unless it stopped the iteration, the G pass (r'.s in q0)
                ns.phase = PH_P2;
                transition<MIXED>(S, ns, q1, 0.0, a.o, a.gs);
                if (ns.phase == PH_APPLY2) transition<MIXED>(S, ns, q0, 0.0, a.o, a.gs);
              } else {
                transition<MIXED>(S, ns, q0, q1, a.o, a.gs);
              }
              nxt[sid] = ns;
              if (ns.phase == PH_DONE) cur[sid] = ns;
              a.cnt[sid] = 0u;
            }
          }
        }
        __syncthreads();
      }
    }
    ++slots;
    const int ex = grid_barrier(a.gs, gridDim.x, a.limit_ns, &sflag);
    if (ex || slots >= a.max_slots) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.gs->slot = slot0 + slots;
}

// Item dependencies of a fused step: for every item, the range of producer
// items (G^T pass) whose rows hold the columns that the item's rows of the
// consumer matrix (G) reach.  One block per item: the column range of the
// item's CSR entries, then the producer items by binary search over their
// first rows.  Rows come in CSR row groups (sell 0) or 32-row slices (sell 1).
__global__ void deps_kernel(const int32_t* __restrict__ rp_c, const int32_t* __restrict__ ci_c,
                            const int32_t* __restrict__ tiles_c, int nt_c, int k_c, int fmt_c,
                            const int32_t* __restrict__ tiles_p, int nt_p, int k_p, int fmt_p, int nitems,
                            int64_t n, int32_t* __restrict__ dep, int all) {
  __shared__ int smin[kBlock / 32], smax[kBlock / 32];
  auto row_of = [n](const int32_t* tiles, int g, int fmt) -> int64_t {
    const int64_t r = (int64_t)__ldg(tiles + g) * rows_per_unit(fmt);
    return r < n ? r : n;
  };
  for (int v = blockIdx.x; v < nitems; v += gridDim.x) {
    if (all) {
      if (threadIdx.x == 0) {
        dep[2 * v] = 0;
        dep[2 * v + 1] = nitems - 1;
      }
      continue;
    }
    const int g0 = v * k_c;
    const int g1 = min(g0 + k_c, nt_c);
    int lo = INT32_MAX, hi = -1;
    if (g0 < g1) {
      const int64_t r0 = row_of(tiles_c, g0, fmt_c), r1 = row_of(tiles_c, g1, fmt_c);
      if (r0 < r1) {
        const int64_t e0 = __ldg(rp_c + r0), e1 = __ldg(rp_c + r1);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          const int c = __ldg(ci_c + e);
          lo = min(lo, c);
          hi = max(hi, c);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
      smin[threadIdx.x >> 5] = lo;
      smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kBlock / 32; ++w) {
        lo = min(lo, smin[w]);
        hi = max(hi, smax[w]);
      }
      int u_lo = 0, u_hi = -1;  // empty range: nothing to wait for
      if (hi >= 0) {
        // last producer item whose first row is <= c
        auto item_of = [&](int c) {
          int a = 0, b = nitems - 1;
          while (a < b) {
            const int mid = (a + b + 1) >> 1;
            const int g = min(mid * k_p, nt_p);
            if (row_of(tiles_p, g, fmt_p) <= c) a = mid; else b = mid - 1;
          }
          return a;
        };
        u_lo = item_of(lo);
        u_hi = item_of(hi);
      }
      dep[2 * v] = u_lo;
      dep[2 * v + 1] = u_hi;
    }
    __syncthreads();
  }
}

// ---- true residual ||b - A x|| / ||b|| (float64, deterministic) ----
__global__ void true_residual_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const double* __restrict__ v, const double* __restrict__ b,
                                     const double* __restrict__ x, int64_t n, double* part) {
  __shared__ double red[32];
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s = __fma_rn(v[e], x[ci[e]], s);
    const double r = b[i] - s;
    rr += r * r;
    bb += b[i] * b[i];
  }
  rr = block_sum(rr, red);
  bb = block_sum(bb, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rr;
    part[2 * blockIdx.x + 1] = bb;
  }
}

// Body tail of the graph-resident solve loop: counts the persistent launch
// that just ended and decides on the device whether another one runs.
__global__ void engine_continue_kernel(GridSync* gs, int64_t slot_cap, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int live = *(volatile int*)&gs->live;
    const int err = *(volatile int*)&gs->err;
    const int slot = *(volatile int*)&gs->slot;
    gs->pad[0] += 1;
    cudaGraphSetConditional(h, (live > 0 && err == 0 && (int64_t)slot < slot_cap) ? 1u : 0u);
  }
}

// Between launches of a batch: the launch table dealt again over the systems
// still running (the same order by size, the same snake), so that members
// that finished leave neither holes nor idle blocks.  One block; the items
// (ord_sys, ord_tile: every member's items in order of decreasing size) are
// ranked among the live ones by a block-wide scan.  Which block runs an item
// does not change its arithmetic.
__global__ void __launch_bounds__(1024) redeal_kernel(GridSync* gs, const EngState* st0, const EngState* st1,
                                                      const int32_t* __restrict__ ord_sys,
                                                      const int32_t* __restrict__ ord_tile, int64_t items, int grid,
                                                      int32_t nsys, int64_t cap, int32_t* item_sys,
                                                      int32_t* item_tile) {
  __shared__ int wsum[32];
  __shared__ int64_t base;
  const int slot = *(volatile int*)&gs->slot;
  const EngState* cur = (slot & 1) ? st1 : st0;  // the states the next launch starts from
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < items; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    int sid = -1, live = 0;
    if (i < items) {
      sid = __ldg(ord_sys + i);
      if (sid < 0 || sid >= nsys) {
        atomicCAS(&gs->err, 0, kErrTable);
        sid = -1;
      } else {
        live = __ldcg(&cur[sid].phase) != PH_DONE ? 1 : 0;
      }
    }
    // exclusive rank of this item among the chunk's live items
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    const int below = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < wid) before += wsum[w];
      total += wsum[w];
    }
    if (live) {
      const int64_t pos = snake_pos(base + before + below, grid);
      if (pos < cap) {
        item_sys[pos] = sid;
        item_tile[pos] = __ldg(ord_tile + i);
      } else {
        atomicCAS(&gs->err, 0, kErrTable);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  // holes of the last round: the blocks it does not reach
  const int64_t nl = base;
  const int64_t rounds = (nl + grid - 1) / grid;
  const int rem = (int)(nl - (rounds > 0 ? (rounds - 1) * grid : 0));  // items in the last round
  if (rounds > 0 && rem < grid && rounds * grid <= cap) {
    const int64_t r = rounds - 1;
    for (int b = threadIdx.x; b < grid; b += blockDim.x) {
      const bool hole = (r & 1) ? (b < grid - rem) : (b >= rem);
      if (hole) item_sys[r * grid + b] = -1;
    }
  }
  if (threadIdx.x == 0) gs->npos = (int)(rounds * grid <= cap ? rounds * grid : 0);
}

template <class VT, class GT, bool MIXED>
const void* kernel_ptr(int kv) {
  if (kv == 0) return reinterpret_cast<const void*>(&engine_kernel<VT, GT, MIXED, 0>);
  if (kv == 1) return reinterpret_cast<const void*>(&engine_kernel<VT, GT, MIXED, 1>);
  return reinterpret_cast<const void*>(&engine_kernel<VT, GT, MIXED, 2>);
}

const void* select_kernel(bool mixed, int gtype, int kv) {
  if (!mixed) {
    if (gtype == SPAI_F64) return kernel_ptr<double, double, false>(kv);
    if (gtype == SPAI_F32) return kernel_ptr<double, float, false>(kv);
    return nullptr;
  }
  if (gtype == SPAI_F32) return kernel_ptr<float, float, true>(kv);
  if (gtype == SPAI_BF16) return kernel_ptr<float, __nv_bfloat16, true>(kv);
  if (gtype == SPAI_F16) return kernel_ptr<float, __half, true>(kv);
  return nullptr;
}

}  // namespace

// Dynamic shared memory of a launch: the SELL-32 ring, the CSR ring with its
// product buffers when a member streams CSR groups (csr_ring), and the
// direct path's buffer over stage 0.  A launch without CSR groups leaves the
// rest of the SM's shared-memory/L1 array to L1, where the vector gathers hit.
size_t engine_smem_bytes(bool mixed, bool csr_ring = true) {
  auto mx = [](size_t x, size_t y) { return x > y ? x : y; };
  const size_t prod = (size_t)kCap * sizeof(double);
  if (mixed) {
    using L = StageLayout<float>;
    const size_t csr = (size_t)L::kCsrStages * L::kStageBytes + (size_t)(kBlock / 32) * kWarpE * sizeof(float);
    return mx(mx((size_t)L::kStages * L::kStageBytes, csr_ring ? csr : 0), prod);
  }
  using L = StageLayout<double>;
  const size_t csr = (size_t)L::kCsrStages * L::kStageBytes + (size_t)(kBlock / 32) * kWarpE * sizeof(double);
  return mx(mx((size_t)L::kStages * L::kStageBytes, csr_ring ? csr : 0), prod);
}

bool engine_groups_fit(int32_t max_row) { return max_row >= 1 && max_row <= kCap / 2; }

// Groups per work item: a system alone has its items dealt one per block per
// round, so pick the K minimising  rounds * (K * t_group + t_item)  with
// rounds = ceil(items / grid), t_item ~ 3 t_group of fixed per-item cost.  Depends only on the
// system's group count and the kernel's co-resident grid.
int engine_items_k(int ngroups, int grid) {
  if (ngroups <= 1 || grid <= 0) return 1;
  int best_k = 1;
  double best = 1e300;
  const int kmax = ngroups < kMaxK ? ngroups : kMaxK;
  for (int k = 1; k <= kmax; ++k) {
    const int64_t items = (ngroups + k - 1) / k;
    const int64_t rounds = (items + grid - 1) / grid;
    const double t = (double)rounds * (k + 3.0);
    if (t < best - 1e-9) { best = t; best_k = k; }
    if (items <= 1) break;
  }
  return best_k;
}

// The tuned multiple of the heuristic K (2^log2), kept within [1, min(ngroups, kMaxK)].
int engine_scale_k(int k, int log2, int ngroups) {
  int64_t v = k;
  if (log2 > 0) v <<= (log2 > 8 ? 8 : log2);
  if (log2 < 0) v >>= (-log2 > 8 ? 8 : -log2);
  const int64_t hi = ngroups < kMaxK ? (ngroups > 0 ? ngroups : 1) : kMaxK;
  if (v > hi) v = hi;
  if (v < 1) v = 1;
  return (int)v;
}

// Tile size for a matrix whose longest row has max_row entries: binning rows
// by their first entry gives tiles of at most tile_nnz + max_row - 1 entries,
// so tile_nnz = kCap - max_row + 1 makes every tile one staging group.
int engine_tile_nnz(int32_t max_row) {
  if (max_row < 1) max_row = 1;
  if (max_row > kCap / 2) return kCap / 2;
  return kCap - max_row + 1;
}

size_t engine_work_bytes(int64_t n, bool mixed, bool pair) {
  const size_t vsz = mixed ? sizeof(float) : sizeof(double);
  const size_t stride = ((n * vsz + 255) / 256) * 256;
  return stride * ((mixed ? 9 : 7) + (pair ? 2 : 0)) + 256;  // paired: r and d buffers twice as long
}

// A set of systems advanced together by the persistent kernel.  Members keep
// their own state across launches; the set can be replaced between launches
// (the server admits and retires systems that way).
class EngineBatch {
 public:
  struct Member {
    SystemData* S;
    PrecondData* M;
    const double* b;
    double* x;
    void* work;              // engine_work_bytes(n, mixed, pair) bytes of device memory
    int32_t pair;            // vector layout of `work` (the system's schedule when the solve began)
    double* history;
    int64_t history_len;
    double* lanczos;
    int64_t lanczos_len;
    EngState st;             // state to start from (fresh or carried over)
  };

  static EngState fresh_state(bool mixed) {
    EngState st;
    memset(&st, 0, sizeof(st));
    st.phase = mixed ? PH_RESID64 : PH_RESID0;
    st.status = SPAI_OK;
    return st;
  }

  int init(bool mixed, int gtype, const spai_pcg_opts& o, cudaStream_t s) {
    mixed_ = mixed;
    s_ = s;
    opts_ = o;
    for (int kv = 0; kv < 3; ++kv) kfns_[kv] = select_kernel(mixed, gtype, kv);
    kfn_csr_ = kfns_[2];
    kfn_sell_ = kfns_[0];
    kfn_ = kfn_csr_;
    if (!kfn_)
      return set_error(SPAI_ERR_INVALID, mixed ? "mixed precision needs G stored as F32, BF16 or F16"
                                               : "float64 precision needs G stored as F64 or F32");
    smem_max_ = engine_smem_bytes(mixed);
    smem_ = smem_max_;
    int per_sell = 0;
    per_sm_ = 1 << 30;
    for (int kv = 0; kv < 3; ++kv) {
      SPAI_CUDA(cudaFuncSetAttribute(kfns_[kv], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max_));
      SPAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sell, kfns_[kv], kBlock, smem_max_));
      if (per_sell < per_sm_) per_sm_ = per_sell;  // one grid for every variant
    }
    if (per_sm_ < 1) return set_error(SPAI_ERR_CUDA, "engine kernel cannot be resident");
    grid_max_ = per_sm_ * num_sms();
    return SPAI_OK;
  }

  int grid_max() const { return grid_max_; }

  // Builds the launch tables for `members` (a member whose state is DONE
  // takes no work).  grid_override > 0 caps the grid.
  int set_members(const std::vector<Member>& members, int grid_override = 0) {
    int rc;
    const int nsys = (int)members.size();
    nsys_ = nsys;
    std::vector<EngSys> hs(nsys);
    int64_t items = 0, chunks = 0, nmax = 0;
    int live = 0;
    bool csr_ring = false;  // a member streams CSR groups through the ring (or uses the block layout)
    bool rmap = false;      // a member has row-mapped SELL-32 slices
    for (int i = 0; i < nsys; ++i) {
      const Member& mb = members[i];
      SystemData& A = *mb.S;
      PrecondData& P = *mb.M;
      const int tn = A.tile_nnz;
      EngSys& e = hs[i];
      memset(&e, 0, sizeof(e));
      e.rp[MAT_A] = A.rowptr.as<int32_t>();
      e.a_ci64 = A.colidx.as<int32_t>();
      e.a_v64 = A.val64.as<double>();
      e.rp[MAT_GT] = P.P->gt_rp();
      e.rp[MAT_G] = P.P->g_rp();
      const int fits = (engine_groups_fit(A.max_row) && A.staged) ? 1 : 0;
      // SELL-32 where the matrix has the layout and the schedule asks for it
      // (all three share one choice, so a system's arithmetic depends on its
      // schedule only); the group size scales like the CSR one
      // the 3 x 3 block layout where A (and G on its pattern) have it and the
      // schedule asks for it, else SELL-32, else CSR row groups
      const bool blk_a = A.block && A.bsell_a.nslices > 0 && A.bsell_v64.p;
      const bool blk_g = A.block && P.P->bsell.nslices > 0 && P.bsell_g.p && P.bsell_gt.p;
      const bool sell_a = !blk_a && A.sell && A.sell_a.nslices > 0 && A.sell_v64.p;
      const bool sell_g = !blk_g && A.sell && P.P->sell.nslices > 0 && P.sell_g.p && P.sell_gt.p;
      const int32_t tblk = (tn + 8) / 9 > 1 ? (tn + 8) / 9 : 1;  // blocks per group (about tn values)
      const int32_t t0 = engine_tile_nnz(A.max_row);
      auto sell_tile = [&](int32_t width) {
        const int64_t tmax = (int64_t)kCap + 1 - 32 * (int64_t)width;
        int64_t t = tmax * tn / (t0 > 0 ? t0 : 1);
        if (t > tmax) t = tmax;
        return (int32_t)(t < 1 ? 1 : t);
      };
      if (blk_a) {
        e.fmt[MAT_A] = 2;
        e.sptr[MAT_A] = A.bsell_a.sptr.as<int32_t>();
        e.ci[MAT_A] = A.bsell_a.ci.as<int32_t>();
        e.val[MAT_A] = mixed_ ? (const void*)A.bsell_v32.p : (const void*)A.bsell_v64.p;
        if ((rc = build_tiles(e.sptr[MAT_A], A.bsell_a.nslices, A.bsell_a.total, tblk, A.tiles, s_))) return rc;
      } else if (sell_a) {
        e.fmt[MAT_A] = 1;
        e.sptr[MAT_A] = A.sell_a.sptr.as<int32_t>();
        e.srow[MAT_A] = A.sell_a.row_map();
        e.ci[MAT_A] = A.sell_a.ci.as<int32_t>();
        e.val[MAT_A] = mixed_ ? (const void*)A.sell_v32.p : (const void*)A.sell_v64.p;
        if ((rc = build_tiles(e.sptr[MAT_A], A.sell_a.nslices, A.sell_a.total, sell_tile(A.sell_a.max_width),
                              A.tiles, s_)))
          return rc;
      } else {
        e.ci[MAT_A] = A.colidx.as<int32_t>();
        e.val[MAT_A] = mixed_ ? (const void*)A.val32.p : (const void*)A.val64.p;
        if ((rc = build_tiles(A.rowptr.as<int32_t>(), A.n, A.nnz, tn, A.tiles, s_))) return rc;
      }
      if (blk_g) {
        const SellData& L = P.P->bsell;
        e.fmt[MAT_GT] = e.fmt[MAT_G] = 2;
        e.sptr[MAT_GT] = e.sptr[MAT_G] = L.sptr.as<int32_t>();
        e.ci[MAT_GT] = e.ci[MAT_G] = L.ci.as<int32_t>();
        e.val[MAT_GT] = P.bsell_gt.p;
        e.val[MAT_G] = P.bsell_g.p;
        if ((rc = build_tiles(L.sptr.as<int32_t>(), L.nslices, L.total, tblk, P.gt_tiles, s_))) return rc;
        if ((rc = build_tiles(L.sptr.as<int32_t>(), L.nslices, L.total, tblk, P.g_tiles, s_))) return rc;
      } else if (sell_g) {
        const SellData& L = P.P->sell;
        const int32_t tg = sell_tile(L.max_width);
        e.fmt[MAT_GT] = e.fmt[MAT_G] = 1;
        e.sptr[MAT_GT] = e.sptr[MAT_G] = L.sptr.as<int32_t>();
        e.srow[MAT_GT] = e.srow[MAT_G] = L.row_map();
        e.ci[MAT_GT] = e.ci[MAT_G] = L.ci.as<int32_t>();
        e.val[MAT_GT] = P.sell_gt.p;
        e.val[MAT_G] = P.sell_g.p;
        if ((rc = build_tiles(L.sptr.as<int32_t>(), L.nslices, L.total, tg, P.gt_tiles, s_))) return rc;
        if ((rc = build_tiles(L.sptr.as<int32_t>(), L.nslices, L.total, tg, P.g_tiles, s_))) return rc;
      } else {
        e.ci[MAT_GT] = P.P->gt_ci();
        e.val[MAT_GT] = P.gt_val.p;
        e.ci[MAT_G] = P.P->g_ci();
        e.val[MAT_G] = P.g_val.p;
        if ((rc = build_tiles(P.P->gt_rp(), P.P->n, P.P->nnz, tn, P.gt_tiles, s_))) return rc;
        if ((rc = build_tiles(P.P->g_rp(), P.P->n, P.P->nnz, tn, P.g_tiles, s_))) return rc;
      }
      e.tiles[MAT_A] = A.tiles.starts.as<int32_t>();
      e.tiles[MAT_GT] = P.gt_tiles.starts.as<int32_t>();
      e.tiles[MAT_G] = P.g_tiles.starts.as<int32_t>();
      e.ntiles[MAT_A] = A.tiles.ntiles;
      e.ntiles[MAT_GT] = P.gt_tiles.ntiles;
      e.ntiles[MAT_G] = P.g_tiles.ntiles;
      int ng = 0;
      for (int mm = 0; mm < 3; ++mm) {
        e.fits[mm] = e.fmt[mm] ? 1 : fits;
        if (e.ntiles[mm] > ng) ng = e.ntiles[mm];
        if ((!e.fmt[mm] && e.fits[mm]) || e.fmt[mm] == 2) csr_ring = true;  // the full kernel
        if (e.srow[mm]) rmap = true;
      }
      if (mb.pair) rmap = true;  // paired vectors: variant 1 or 2
      // work items depend only on the system and the kernel's full grid, so a
      // system's reductions are identical alone and in any batch
      const int kg = engine_scale_k(engine_items_k(ng, grid_max_), A.items_log2, ng);
      e.nitems = (ng + kg - 1) / kg;
      for (int mm = 0; mm < 3; ++mm) e.kgroups[mm] = (e.ntiles[mm] + e.nitems - 1) / e.nitems;
      e.fuse = A.fuse ? 1 : 0;
      e.item_base = (int32_t)items;
      e.chunk_base = (int32_t)chunks;
      items += e.nitems;
      chunks += (e.nitems + kChunk - 1) / kChunk;
      e.n = A.n;
      e.eps = P.eps;
      e.b = mb.b;
      e.x = mb.x;
      const size_t vsz = mixed_ ? sizeof(float) : sizeof(double);
      const size_t stride = ((A.n * vsz + 255) / 256) * 256;
      char* base = static_cast<char*>(mb.work);
      if (mb.pair) {  // pair buffers (q, r[0]), (q, r[1]), (s, d[0]), (s, d[1]) of 2n values each
        e.pair = 1;
        e.r[0] = base + vsz; e.r[1] = base + 2 * stride + vsz;
        e.d[0] = base + 4 * stride + vsz; e.d[1] = base + 6 * stride + vsz;
        e.t = base + 8 * stride;
        if (mixed_) { e.e = base + 9 * stride; e.rin = base + 10 * stride; }
      } else {
        e.r[0] = base; e.r[1] = base + stride;
        e.d[0] = base + 2 * stride; e.d[1] = base + 3 * stride;
        e.q = base + 4 * stride; e.t = base + 5 * stride; e.s = base + 6 * stride;
        if (mixed_) { e.e = base + 7 * stride; e.rin = base + 8 * stride; }
      }
      e.history = mb.history;
      e.history_len = mb.history_len;
      e.lanczos = mb.lanczos;
      e.lanczos_len = mb.lanczos_len;
      if (A.n > nmax) nmax = A.n;
      if (mb.st.phase != PH_DONE) ++live;
    }
    if (items >= INT32_MAX) return set_error(SPAI_ERR_INVALID, "too many work items");
    smem_ = engine_smem_bytes(mixed_, csr_ring);
    kfn_ = kfns_[csr_ring ? 2 : (rmap ? 1 : 0)];
    int grid = grid_max_;
    if (grid_override > 0 && grid_override < grid) grid = grid_override;
    if (grid > items) grid = (int)items;
    if (grid < 1) grid = 1;
    // Positions of the items in the launch table: block b runs positions b,
    // b + grid, b + 2 grid, ...  Items are dealt in order of decreasing size
    // (entries of the three matrices in their groups) in a snake, blocks 0 ..
    // grid - 1 and then grid - 1 .. 0, so that members of very different
    // sizes load every block about equally; holes of the last round hold
    // system -1.  Which block runs an item does not change its arithmetic.
    // One system alone in at most one round keeps item v at position v.
    const int64_t npos = deal_positions(items, grid);
    if (npos >= INT32_MAX) return set_error(SPAI_ERR_INVALID, "too many work items");
    std::vector<int32_t> isys(npos, -1), itile(npos, 0), osys, otile;
    {
      std::vector<double> w(items);
      for (int i = 0; i < nsys; ++i) {
        const EngSys& e = hs[i];
        const double ent[3] = {(double)members[i].S->nnz, (double)members[i].M->P->nnz,
                               (double)members[i].M->P->nnz};
        for (int v = 0; v < e.nitems; ++v) {
          double wt = 0.0;
          for (int mm = 0; mm < 3; ++mm) {
            const int64_t g = std::min<int64_t>(e.kgroups[mm], (int64_t)e.ntiles[mm] - (int64_t)v * e.kgroups[mm]);
            if (g > 0 && e.ntiles[mm] > 0) wt += (double)g * ent[mm] / e.ntiles[mm];
          }
          w[e.item_base + v] = wt;
        }
      }
      const std::vector<int64_t> ord = deal_order(w);
      std::vector<int32_t> owner(items), idx(items);
      for (int i = 0; i < nsys; ++i)
        for (int v = 0; v < hs[i].nitems; ++v) {
          owner[hs[i].item_base + v] = i;
          idx[hs[i].item_base + v] = v;
        }
      osys.resize(items);
      otile.resize(items);
      for (int64_t j = 0; j < items; ++j) {
        const int64_t pos = snake_pos(j, grid);
        isys[pos] = osys[j] = owner[ord[j]];
        itile[pos] = otile[j] = idx[ord[j]];
      }
    }
    std::vector<EngState> hst(nsys);
    for (int i = 0; i < nsys; ++i) hst[i] = members[i].st;
    const size_t sz_sys = sizeof(EngSys) * nsys, sz_st = sizeof(EngState) * nsys;
    const size_t sz_items = sizeof(int32_t) * npos, sz_part = sizeof(double) * 2 * items;
    const size_t sz_cnt = sizeof(unsigned) * nsys;
    const size_t sz_cpart = sizeof(double) * 2 * chunks, sz_ccnt = sizeof(unsigned) * chunks;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t off_sys = 0, off_st0 = al(sz_sys), off_st1 = off_st0 + al(sz_st), off_is = off_st1 + al(sz_st);
    const size_t off_it = off_is + al(sz_items), off_part = off_it + al(sz_items), off_cnt = off_part + al(sz_part);
    const size_t off_cpart = off_cnt + al(sz_cnt), off_ccnt = off_cpart + al(sz_cpart);
    const size_t off_gs = off_ccnt + al(sz_ccnt), off_flags = off_gs + al(sizeof(GridSync));
    const size_t off_dep = off_flags + al(sizeof(unsigned) * items);
    const size_t off_ord = off_dep + al(sizeof(int32_t) * 2 * items);  // items by size: system, item
    const size_t total = off_ord + 2 * al(sizeof(int32_t) * items);
    if ((rc = tab_.alloc(total, s_))) return rc;
    char* tb = tab_.as<char>();
    SPAI_CUDA(cudaMemsetAsync(tb, 0, total, s_));
    // item dependencies of fused steps (G pass on G^T-pass items)
    for (int i = 0; i < nsys; ++i) {
      EngSys& e = hs[i];
      if (!e.fuse) continue;
      int32_t* dep = reinterpret_cast<int32_t*>(tb + off_dep) + 2 * (size_t)e.item_base;
      e.dep = dep;
      const PrecondData& P = *members[i].M;
      const int dgrid = e.nitems < 4 * num_sms() ? e.nitems : 4 * num_sms();
      // rows sorted by length within windows: an item's rows are no longer a
      // contiguous range, so its G items wait for every G^T item
      const int all = (e.srow[MAT_G] || e.srow[MAT_GT]) ? 1 : 0;
      deps_kernel<<<dgrid, kBlock, 0, s_>>>(P.P->g_rp(), P.P->g_ci(), e.tiles[MAT_G], e.ntiles[MAT_G],
                                            e.kgroups[MAT_G], e.fmt[MAT_G], e.tiles[MAT_GT], e.ntiles[MAT_GT],
                                            e.kgroups[MAT_GT], e.fmt[MAT_GT], e.nitems, e.n, dep, all);
      count_launch();
      SPAI_CUDA(cudaGetLastError());
    }
    SPAI_CUDA(cudaMemcpyAsync(tb + off_sys, hs.data(), sz_sys, cudaMemcpyHostToDevice, s_));
    SPAI_CUDA(cudaMemcpyAsync(tb + off_st0, hst.data(), sz_st, cudaMemcpyHostToDevice, s_));
    SPAI_CUDA(cudaMemcpyAsync(tb + off_st1, hst.data(), sz_st, cudaMemcpyHostToDevice, s_));
    SPAI_CUDA(cudaMemcpyAsync(tb + off_is, isys.data(), sz_items, cudaMemcpyHostToDevice, s_));
    SPAI_CUDA(cudaMemcpyAsync(tb + off_it, itile.data(), sz_items, cudaMemcpyHostToDevice, s_));
    if (items > 0) {
      SPAI_CUDA(cudaMemcpyAsync(tb + off_ord, osys.data(), sizeof(int32_t) * items, cudaMemcpyHostToDevice, s_));
      SPAI_CUDA(cudaMemcpyAsync(tb + off_ord + al(sizeof(int32_t) * items), otile.data(), sizeof(int32_t) * items,
                                cudaMemcpyHostToDevice, s_));
    }
    ord_sys_ = reinterpret_cast<const int32_t*>(tb + off_ord);
    ord_tile_ = reinterpret_cast<const int32_t*>(tb + off_ord + al(sizeof(int32_t) * items));
    items_ = items;
    GridSync g0;
    memset(&g0, 0, sizeof(g0));
    g0.live = live;
    g0.npos = (int)npos;
    SPAI_CUDA(cudaMemcpyAsync(tb + off_gs, &g0, sizeof(g0), cudaMemcpyHostToDevice, s_));
    // host copies must stay alive until the copies ran
    SPAI_CUDA(cudaStreamSynchronize(s_));
    live_ = live;

    memset(&args_, 0, sizeof(args_));
    args_.sys = reinterpret_cast<const EngSys*>(tb + off_sys);
    args_.st0 = reinterpret_cast<EngState*>(tb + off_st0);
    args_.st1 = reinterpret_cast<EngState*>(tb + off_st1);
    args_.nsys = nsys;
    args_.item_sys = reinterpret_cast<const int32_t*>(tb + off_is);
    args_.item_tile = reinterpret_cast<const int32_t*>(tb + off_it);
    args_.n_items = (int32_t)npos;
    args_.partial = reinterpret_cast<double*>(tb + off_part);
    args_.cnt = reinterpret_cast<unsigned*>(tb + off_cnt);
    args_.cpartial = reinterpret_cast<double*>(tb + off_cpart);
    args_.ccnt = reinterpret_cast<unsigned*>(tb + off_ccnt);
    args_.gs = reinterpret_cast<GridSync*>(tb + off_gs);
    args_.flags = reinterpret_cast<unsigned*>(tb + off_flags);
    int64_t max_iter = opts_.max_iter;
    if (max_iter <= 0) {
      max_iter = 10 * nmax;
      if (max_iter > 1000000) max_iter = 1000000;
    }
    max_iter_ = max_iter;
    args_.o.tol2 = opts_.rtol * opts_.rtol;
    const double rel = (opts_.inner_rtol > 0 && opts_.inner_rtol < 1) ? opts_.inner_rtol : 0.1;
    args_.o.reliable2 = rel * rel;
    args_.o.max_iter = max_iter;
    args_.o.period = opts_.replace_period < 0 ? 0 : opts_.replace_period;
    args_.o.criterion = opts_.criterion;
    args_.o.max_outer = opts_.max_outer > 0 ? opts_.max_outer : 0;
    args_.o.mixed = mixed_ ? 1 : 0;
    args_.limit_ns = 2000000000ull;  // 2 s per device-side wait
    grid_ = grid;
    slots_ = 0;
    return SPAI_OK;
  }

  // Runs every remaining phase from one CUDA graph: a while-conditional node
  // whose body is the persistent launch (chunk slots) followed by a one-thread
  // kernel that decides on the device whether another launch is needed, so the
  // batch runs to the end without returning to the host.  Same kernel, same
  // arguments and the same slot sequence as repeated launch() calls.
  int run_graph(int chunk, int64_t slot_cap, cudaEvent_t ev0, cudaEvent_t ev1, double* ms, int* launches) {
    *launches = 0;
    if (live_ <= 0) return SPAI_OK;
    args_.max_slots = chunk;
    struct G {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t e = nullptr;
      ~G() {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
      }
    } gr;
    SPAI_CUDA(cudaGraphCreate(&gr.g, 0));
    cudaGraphConditionalHandle h;
    SPAI_CUDA(cudaGraphConditionalHandleCreate(&h, gr.g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    SPAI_CUDA(cudaGraphAddNode(&loop, gr.g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    void* kargs[] = {&args_};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void*>(kfn_);
    kp.gridDim = dim3(grid_);
    kp.blockDim = dim3(kBlock);
    kp.sharedMemBytes = (unsigned)smem_;
    kp.kernelParams = kargs;
    cudaGraphNode_t kn;
    SPAI_CUDA(cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp));
    cudaKernelNodeAttrValue coop;
    memset(&coop, 0, sizeof(coop));
    coop.cooperative = 1;
    SPAI_CUDA(cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeCooperative, &coop));
    GridSync* gs = args_.gs;
    void* cargs[] = {&gs, &slot_cap, &h};
    cudaKernelNodeParams cpk;
    memset(&cpk, 0, sizeof(cpk));
    cpk.func = reinterpret_cast<void*>(&engine_continue_kernel);
    cpk.gridDim = dim3(1);
    cpk.blockDim = dim3(32);
    cpk.kernelParams = cargs;
    cudaGraphNode_t prev = kn;
    int32_t* item_sys = const_cast<int32_t*>(args_.item_sys);
    int32_t* item_tile = const_cast<int32_t*>(args_.item_tile);
    EngState* st0 = args_.st0;
    EngState* st1 = args_.st1;
    const EngState* cst0 = st0;
    const EngState* cst1 = st1;
    const int32_t* osys = ord_sys_;
    const int32_t* otile = ord_tile_;
    int64_t nit = items_;
    int grid = grid_;
    int32_t nsys = nsys_;
    int64_t cap = args_.n_items;  // positions the table holds
    void* rargs[] = {&gs, &cst0, &cst1, &osys, &otile, &nit, &grid, &nsys, &cap, &item_sys, &item_tile};
    if (nsys_ > 1 && items_ > 0) {  // members finish at different times: deal the live ones again
      cudaKernelNodeParams rk;
      memset(&rk, 0, sizeof(rk));
      rk.func = reinterpret_cast<void*>(&redeal_kernel);
      rk.gridDim = dim3(1);
      rk.blockDim = dim3(1024);
      rk.kernelParams = rargs;
      cudaGraphNode_t rn;
      SPAI_CUDA(cudaGraphAddKernelNode(&rn, body, &kn, 1, &rk));
      prev = rn;
    }
    cudaGraphNode_t cn;
    SPAI_CUDA(cudaGraphAddKernelNode(&cn, body, &prev, 1, &cpk));
    SPAI_CUDA(cudaGraphInstantiate(&gr.e, gr.g, 0));
    if (ev0) SPAI_CUDA(cudaEventRecord(ev0, s_));
    SPAI_CUDA(cudaGraphLaunch(gr.e, s_));
    if (ev1) SPAI_CUDA(cudaEventRecord(ev1, s_));
    GridSync gh;
    SPAI_CUDA(cudaMemcpyAsync(&gh, args_.gs, sizeof(gh), cudaMemcpyDeviceToHost, s_));
    SPAI_CUDA(cudaStreamSynchronize(s_));
    if (ev0 && ev1 && ms) {
      float f = 0.f;
      SPAI_CUDA(cudaEventElapsedTime(&f, ev0, ev1));
      *ms += f;
    }
    *launches = gh.pad[0];
    count_launch(2 * gh.pad[0]);
    slots_ = gh.slot;
    live_ = gh.live;
    if (gh.err == kErrTable) return set_error(SPAI_ERR_INVALID, "engine: a launch-table entry was out of range");
    if (gh.err) return set_error(SPAI_ERR_TIMEOUT, "engine: a bounded device wait timed out");
    return SPAI_OK;
  }

  int64_t max_iter() const { return max_iter_; }
  int live() const { return live_; }
  int64_t slots() const { return slots_; }

  // One persistent launch of at most max_slots phases; *ms = its device time
  // when events are given.
  int launch(int max_slots, cudaEvent_t ev0, cudaEvent_t ev1, double* ms) {
    if (live_ <= 0) return SPAI_OK;
    args_.max_slots = max_slots;
    void* kargs[] = {&args_};
    if (ev0) SPAI_CUDA(cudaEventRecord(ev0, s_));
    SPAI_CUDA(cudaLaunchCooperativeKernel(kfn_, dim3(grid_), dim3(kBlock), kargs, smem_, s_));
    count_launch();
    if (ev1) SPAI_CUDA(cudaEventRecord(ev1, s_));
    GridSync gh;
    SPAI_CUDA(cudaMemcpyAsync(&gh, args_.gs, sizeof(gh), cudaMemcpyDeviceToHost, s_));
    SPAI_CUDA(cudaStreamSynchronize(s_));
    if (ev0 && ev1 && ms) {
      float f = 0.f;
      SPAI_CUDA(cudaEventElapsedTime(&f, ev0, ev1));
      *ms += f;
    }
    slots_ = gh.slot;
    live_ = gh.live;
    if (gh.err == kErrTable) return set_error(SPAI_ERR_INVALID, "engine: a launch-table entry was out of range");
    if (gh.err) return set_error(SPAI_ERR_TIMEOUT, "engine: a bounded device wait timed out");
    return SPAI_OK;
  }

  // Current state of every member.
  int read_states(std::vector<EngState>& out) {
    out.resize(nsys_);
    SPAI_CUDA(cudaMemcpyAsync(out.data(), (slots_ & 1) ? args_.st1 : args_.st0, sizeof(EngState) * nsys_,
                              cudaMemcpyDeviceToHost, s_));
    SPAI_CUDA(cudaStreamSynchronize(s_));
    return SPAI_OK;
  }

 private:
  bool mixed_ = false;
  cudaStream_t s_ = nullptr;
  spai_pcg_opts opts_;
  const void* kfns_[3] = {nullptr, nullptr, nullptr};  // kernel variants 0, 1, 2
  const void* kfn_ = nullptr;  // this launch's kernel
  const void* kfn_csr_ = nullptr;
  const void* kfn_sell_ = nullptr;
  size_t smem_ = 0, smem_max_ = 0;  // this launch's dynamic shared memory; the largest
  int per_sm_ = 0, grid_max_ = 0, grid_ = 0, nsys_ = 0, live_ = 0;
  int64_t max_iter_ = 0, slots_ = 0;
  DevMem tab_;
  EngArgs args_;
  const int32_t* ord_sys_ = nullptr;   // every member's items in order of decreasing size
  const int32_t* ord_tile_ = nullptr;
  int64_t items_ = 0;
};

// ||b - A x|| / ||b|| for each system (float64, deterministic).
int engine_true_residuals(int nsys, SystemData* const* S, const double* const* b, double* const* x, double* out,
                          cudaStream_t s) {
  const int rgrid = 2 * num_sms();
  DevMem part;
  int rc;
  if ((rc = part.alloc(sizeof(double) * 2 * rgrid * nsys, s))) return rc;
  for (int i = 0; i < nsys; ++i) {
    true_residual_kernel<<<rgrid, 256, 0, s>>>(S[i]->rowptr.as<int32_t>(), S[i]->colidx.as<int32_t>(),
                                               S[i]->val64.as<double>(), b[i], x[i], S[i]->n,
                                               part.as<double>() + 2 * rgrid * i); count_launch();
    SPAI_CUDA(cudaGetLastError());
  }
  std::vector<double> hp(2 * rgrid * nsys);
  SPAI_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < nsys; ++i) {
    double rr = 0, bb = 0;
    for (int k = 0; k < rgrid; ++k) { rr += hp[2 * rgrid * i + 2 * k]; bb += hp[2 * rgrid * i + 2 * k + 1]; }
    out[i] = bb > 0 ? sqrt(rr / bb) : 0.0;
  }
  return SPAI_OK;
}

int engine_check_opts(const spai_pcg_opts* o) {
  if (o->precision != SPAI_PREC_F64 && o->precision != SPAI_PREC_MIXED)
    return set_error(SPAI_ERR_INVALID, "unknown precision");
  if (o->criterion != SPAI_CRIT_RESIDUAL && o->criterion != SPAI_CRIT_PRECOND)
    return set_error(SPAI_ERR_INVALID, "unknown criterion");
  if (!(o->rtol >= 0.0)) return set_error(SPAI_ERR_INVALID, "rtol must be >= 0");
  return SPAI_OK;
}

void engine_fill_result(const EngState& f, double true_rel, double engine_ms, int64_t slots, int launches,
                        spai_pcg_result& r) {
  memset(&r, 0, sizeof(r));
  r.iters = f.iter;
  r.outer_iters = f.outer;
  r.status = (f.phase == PH_DONE) ? f.status : SPAI_ERR_NOT_CONVERGED;
  r.true_rel_res = true_rel;
  r.rec_rel_res = f.bb > 0 ? sqrt(f.rr / f.bb) : 0.0;
  r.history_written = f.hist_n;
  r.engine_ms = engine_ms;
  r.slots = slots;
  r.launches = launches;
}

// Runs PCG on nsys systems in one persistent launch sequence.
int engine_run(int nsys, SystemData* const* S, PrecondData* const* M, const double* const* b, double* const* x,
               const spai_pcg_opts* o, spai_pcg_result* res, cudaStream_t s, int grid_override, int use_graph) {
  if (nsys <= 0) return set_error(SPAI_ERR_INVALID, "nsys must be positive");
  int rc;
  if ((rc = engine_check_opts(o))) return rc;
  const bool mixed = o->precision == SPAI_PREC_MIXED;
  const int gtype = M[0]->gtype;
  for (int i = 0; i < nsys; ++i) {
    if (!S[i] || !M[i] || !b[i] || !x[i]) return set_error(SPAI_ERR_INVALID, "null system, preconditioner or vector");
    if (M[i]->gtype != gtype) return set_error(SPAI_ERR_INVALID, "all preconditioners of a batch need one G type");
    if (M[i]->P->n != S[i]->n) return set_error(SPAI_ERR_SHAPE, "G and A sizes differ (system %d)", i);
  }
  EngineBatch B;
  if ((rc = B.init(mixed, gtype, *o, s))) return rc;
  std::vector<DevMem> ws(nsys);
  std::vector<EngineBatch::Member> mem(nsys);
  for (int i = 0; i < nsys; ++i) {
    if ((rc = ws[i].alloc(engine_work_bytes(S[i]->n, mixed, S[i]->pair != 0), s))) return rc;
    EngineBatch::Member& m = mem[i];
    m.S = S[i];
    m.M = M[i];
    m.b = b[i];
    m.x = x[i];
    m.work = ws[i].p;
    m.pair = S[i]->pair;
    m.history = (nsys == 1 && o->record_history) ? o->history : nullptr;
    m.history_len = (nsys == 1 && o->record_history) ? o->history_len : 0;
    m.lanczos = (nsys == 1 && o->lanczos && o->lanczos_len > 0) ? o->lanczos : nullptr;
    m.lanczos_len = m.lanczos ? o->lanczos_len : 0;
    m.st = EngineBatch::fresh_state(mixed);
  }
  if ((rc = B.set_members(mem, grid_override))) return rc;
  const int64_t slot_cap = 8 * B.max_iter() + 64;
  // a batch returns to the re-deal every 128 slots (members finish at
  // different times); one system alone keeps its table for 3000
  const int chunk = nsys > 1 ? 128 : 3000;
  int launches = 0;
  double engine_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SPAI_CUDA(cudaEventCreate(&ev0));
  SPAI_CUDA(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } evg{ev0, ev1};
  if (use_graph) {
    if ((rc = B.run_graph(chunk, slot_cap, ev0, ev1, &engine_ms, &launches))) return rc;
  } else {
    while (B.live() > 0) {
      const int64_t left = slot_cap - B.slots();
      if (left <= 0) break;
      if ((rc = B.launch((int)(left < chunk ? left : chunk), ev0, ev1, &engine_ms))) return rc;
      ++launches;
    }
  }
  std::vector<EngState> fin;
  if ((rc = B.read_states(fin))) return rc;
  std::vector<double> tr(nsys);
  if ((rc = engine_true_residuals(nsys, S, b, x, tr.data(), s))) return rc;
  int first_bad = SPAI_OK;
  for (int i = 0; i < nsys; ++i) {
    engine_fill_result(fin[i], tr[i], engine_ms, B.slots(), launches, res[i]);
    if (mem[i].lanczos) res[i].lanczos_written = fin[i].iter < mem[i].lanczos_len ? fin[i].iter : mem[i].lanczos_len;
    if (res[i].status != SPAI_OK && first_bad == SPAI_OK) first_bad = res[i].status;
  }
  if (first_bad != SPAI_OK)
    set_error(first_bad, "pcg: %s", first_bad == SPAI_ERR_BREAKDOWN ? "breakdown" : "not converged");
  return first_bad;
}

namespace {
__global__ void tune_rhs_kernel(double* b, double* x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    b[i] = 1.0 + 0.25 * (double)(i % 5);
    x[i] = 0.0;
  }
}
}  // namespace

// Schedule autotuner: times short solves (a fixed right-hand side, rtol 0,
// kTuneIters iterations, best of two runs) of the system with the given
// preconditioner and precision for every candidate schedule -- tile size
// (entries per group) T0, T0/2, T0/4; groups per work item x1/2, x1, x2;
// SELL-32 slices (when the matrices have the layout), TMA-staged CSR groups
// or CSR with direct loads -- and keeps the fastest.  The heuristic
// schedule is kept unless a candidate beats it by more than 3%.
int engine_tune(SystemData* S, PrecondData* M, bool mixed, cudaStream_t s) {
  constexpr int kTuneIters = 12;
  const int32_t t0 = engine_tile_nnz(S->max_row);
  struct Cand { int32_t tile, klog, staged, sell, fuse, block; };
  std::vector<Cand> cands;
  const bool has_sell = S->sell_a.nslices > 0 || M->P->sell.nslices > 0;
  for (int div : {1, 2, 4}) {
    const int32_t t = t0 / div;
    if (div > 1 && t < 256) continue;
    for (int kl : {0, -1, 1}) {
      if (has_sell) cands.push_back(Cand{t, kl, 1, 1, 1, 1});
      for (int st : {1, 0}) {
        if (st == 0 && !engine_groups_fit(S->max_row)) continue;  // direct loads either way
        cands.push_back(Cand{t, kl, st, 0, 1, 1});
      }
    }
  }
  {
    Cand c = cands[0];  // the heuristic schedule with one grid step per pass
    c.fuse = 0;
    cands.push_back(c);
  }
  // systems made of 3 x 3 blocks: the block layout (default) against the scalar ones
  const bool has_blk = S->bsell_a.nslices > 0 || M->P->bsell.nslices > 0;
  for (Cand& c : cands) c.block = 1;
  if (has_blk) {
    const size_t nc = cands.size();
    for (size_t i = 0; i < nc; ++i)
      if (cands[i].tile == t0 && cands[i].fuse) {
        Cand c = cands[i];
        c.block = 0;
        cands.push_back(c);
      }
  }
  DevMem buf;
  int rc;
  if ((rc = buf.alloc(2 * (size_t)S->n * sizeof(double), s))) return rc;
  double* b = buf.as<double>();
  double* x = b + S->n;
  spai_pcg_opts o;
  spai_pcg_opts_default(&o);
  o.rtol = 0.0;
  o.max_iter = kTuneIters;
  o.precision = mixed ? SPAI_PREC_MIXED : SPAI_PREC_F64;
  o.record_history = 0;
  double best_t = 1e300, base_t = 1e300;
  Cand best = cands[0];
  for (const Cand& c : cands) {
    S->tile_nnz = c.tile;
    S->items_log2 = c.klog;
    S->staged = c.staged;
    S->sell = c.sell;
    S->fuse = c.fuse;
    S->block = c.block;
    double t = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      tune_rhs_kernel<<<256, 256, 0, s>>>(b, x, S->n);
      count_launch();
      spai_pcg_result r;
      const double* bc = b;
      rc = engine_run(1, &S, &M, &bc, &x, &o, &r, s, 0, 0);
      if (rc != SPAI_OK && rc != SPAI_ERR_NOT_CONVERGED) return rc;
      if (r.engine_ms < t) t = r.engine_ms;
    }
    if (&c == &cands[0]) base_t = t;
    if (t < best_t) {
      best_t = t;
      best = c;
    }
  }
  if (best_t > 0.97 * base_t) best = cands[0];
  S->tile_nnz = best.tile;
  S->items_log2 = best.klog;
  S->staged = best.staged;
  S->sell = best.sell;
  S->fuse = best.fuse;
  S->block = best.block;
  S->tuned = 1;
  set_error(SPAI_OK, "no error");
  return SPAI_OK;
}

}  // namespace spai

// ---------------------------------------------------------------------------
// Session interface used by the server: a batch whose members carry their
// state (an opaque block of engine_state_bytes()) across launches.
// ---------------------------------------------------------------------------
namespace spai {

struct EngineSession {
  EngineBatch batch;
  bool mixed;
};

size_t engine_state_bytes() { return sizeof(EngState); }

int session_create(bool mixed, int gtype, const spai_pcg_opts& o, cudaStream_t s, EngineSession** out) {
  int rc;
  if ((rc = engine_check_opts(&o))) return rc;
  auto* es = new EngineSession();
  es->mixed = mixed;
  if ((rc = es->batch.init(mixed, gtype, o, s))) {
    delete es;
    return rc;
  }
  *out = es;
  return SPAI_OK;
}

int session_set(EngineSession* es, std::vector<SessionMember>& members) {
  std::vector<EngineBatch::Member> mem(members.size());
  for (size_t i = 0; i < members.size(); ++i) {
    SessionMember& sm = members[i];
    EngineBatch::Member& m = mem[i];
    m.S = sm.S;
    m.M = sm.M;
    m.b = sm.b;
    m.x = sm.x;
    m.work = sm.work;
    m.pair = sm.pair;
    m.history = nullptr;
    m.history_len = 0;
    m.lanczos = nullptr;
    m.lanczos_len = 0;
    if (sm.state.size() == sizeof(EngState)) memcpy(&m.st, sm.state.data(), sizeof(EngState));
    else m.st = EngineBatch::fresh_state(es->mixed);
  }
  return es->batch.set_members(mem);
}

int session_launch(EngineSession* es, int max_slots) { return es->batch.launch(max_slots, nullptr, nullptr, nullptr); }

int session_live(EngineSession* es) { return es->batch.live(); }

int session_read(EngineSession* es, std::vector<SessionMember>& members, std::vector<SessionView>& views) {
  std::vector<EngState> st;
  int rc;
  if ((rc = es->batch.read_states(st))) return rc;
  views.resize(st.size());
  for (size_t i = 0; i < st.size(); ++i) {
    members[i].state.resize(sizeof(EngState));
    memcpy(members[i].state.data(), &st[i], sizeof(EngState));
    views[i].done = st[i].phase == PH_DONE;
    views[i].status = st[i].status;
    views[i].iters = st[i].iter;
    views[i].outer = st[i].outer;
  }
  return SPAI_OK;
}

void session_destroy(EngineSession* es) { delete es; }

}  // namespace spai

// ---------------------------------------------------------------------------
// Allocation-free float64 solve.
//
// For callers that cannot allocate device memory while they solve (for
// example code running under a custom device allocator or a memory budget
// that forbids cudaMalloc), spai_pcg_solve_noalloc takes every matrix as a
// raw device CSR and keeps all of its working memory in one file-scope
// device array of kNoAllocBytes.  That array exists on every GPU that loads
// the library, for the lifetime of the process.  All calls share it: calls
// that overlap on the GPU (other streams, other host threads) race and must
// be serialised by the caller.
// ---------------------------------------------------------------------------
namespace spai {

int launch_validate(const spai_csr* A, int check_sym, int* flags, cudaStream_t s);
std::string validate_flag_text(int f);
int launch_tiles(const int32_t* rowptr, int64_t n, int64_t nnz, int32_t tile_nnz, int32_t ntiles, int32_t* starts,
                 cudaStream_t s);

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;   // 8 MiB of device scratch
constexpr int64_t kNoAllocMaxN = 131072;             // rows at most
constexpr int64_t kNoAllocMaxNnz = int64_t(1) << 22; // stored entries per matrix at most

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array, looked up once per device (the
// symbol's host-side name is not a device address).
int noalloc_scratch_ptr(unsigned char** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  SPAI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(SPAI_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(addr[dev]);
  return SPAI_OK;
}

}  // namespace

}  // namespace spai

extern "C" int spai_pcg_solve_noalloc(const spai_csr* A, const spai_csr* G, const spai_csr* GT, double eps,
                                      const double* b, double* x, const spai_pcg_opts* o, spai_pcg_result* res,
                                      void* stream) {
  using namespace spai;
  if (!A || !G || !GT || !b || !x || !o || !res) return set_error(SPAI_ERR_INVALID, "null argument");
  if (o->precision != SPAI_PREC_F64)
    return set_error(SPAI_ERR_INVALID, "the allocation-free solve runs in float64 only (precision F64)");
  if (o->criterion != SPAI_CRIT_RESIDUAL && o->criterion != SPAI_CRIT_PRECOND)
    return set_error(SPAI_ERR_INVALID, "unknown criterion");
  if (!(o->rtol >= 0.0) || !(eps >= 0.0)) return set_error(SPAI_ERR_INVALID, "rtol and eps must be >= 0");
  const spai_csr* mats[3] = {A, GT, G};
  for (const spai_csr* m : mats) {
    if (m->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A, G and G^T values must be SPAI_F64");
    if (m->n != A->n) return set_error(SPAI_ERR_SHAPE, "A, G and G^T must have the same n");
    if (m->n <= 0 || m->n > kNoAllocMaxN || m->nnz < 0 || m->nnz > kNoAllocMaxNnz)
      return set_error(SPAI_ERR_TOO_LARGE, "allocation-free solve supports n in 1..%lld and nnz <= %lld per matrix",
                       (long long)kNoAllocMaxN, (long long)kNoAllocMaxNnz);
  }
  if (G->nnz != GT->nnz) return set_error(SPAI_ERR_SHAPE, "G and G^T must have the same nnz");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  int rc;
  if ((rc = noalloc_scratch_ptr(&base))) return rc;
  const int64_t n = A->n;

  // kernel and grid
  const void* kfn = select_kernel(false, SPAI_F64, 2);
  const int block = kBlock;
  const size_t smem = engine_smem_bytes(false);
  SPAI_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SPAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, block, smem));
  if (per_sm < 1) return set_error(SPAI_ERR_CUDA, "engine kernel cannot be resident");
  const int grid_max = per_sm * num_sms();

  // scratch layout: [flags 3x2 ints | tiles A, G^T, G | tables | partials | vectors]
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t off = 0;
  const size_t off_flags = off; off += al(6 * sizeof(int));
  SPAI_CUDA(cudaMemsetAsync(base + off_flags, 0, 6 * sizeof(int), s));
  for (int k = 0; k < 3; ++k)
    if ((rc = launch_validate(mats[k], 0, reinterpret_cast<int*>(base + off_flags) + 2 * k, s))) return rc;
  int hf[6];
  SPAI_CUDA(cudaMemcpyAsync(hf, base + off_flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 3; ++k)
    if (hf[2 * k]) return set_error(SPAI_ERR_BAD_CSR, "invalid CSR (%s): %s", k == 0 ? "A" : (k == 1 ? "G^T" : "G"),
                                    validate_flag_text(hf[2 * k]).c_str());
  int32_t max_row = hf[1];
  if (hf[3] > max_row) max_row = hf[3];
  if (hf[5] > max_row) max_row = hf[5];
  const int32_t tn = engine_tile_nnz(max_row);
  int32_t ntl[3];
  size_t off_tiles[3];
  for (int k = 0; k < 3; ++k) {
    int64_t nt = (mats[k]->nnz + tn - 1) / tn;
    if (nt < 1) nt = 1;
    ntl[k] = (int32_t)nt;
    off_tiles[k] = off;
    off += al((nt + 1) * sizeof(int32_t));
  }
  EngSys e;
  memset(&e, 0, sizeof(e));
  for (int k = 0; k < 3; ++k) {
    e.rp[k] = mats[k]->rowptr;
    e.ci[k] = mats[k]->colidx;
    e.val[k] = mats[k]->val;
    e.tiles[k] = reinterpret_cast<const int32_t*>(base + off_tiles[k]);
    e.ntiles[k] = ntl[k];
    e.fits[k] = 0;  // caller arrays carry no alignment padding: direct loads
  }
  e.a_v64 = static_cast<const double*>(A->val);
  e.a_ci64 = A->colidx;
  int ng = ntl[0] > ntl[1] ? ntl[0] : ntl[1];
  if (ntl[2] > ng) ng = ntl[2];
  const int kg = engine_items_k(ng, grid_max);
  e.nitems = (ng + kg - 1) / kg;
  for (int k = 0; k < 3; ++k) e.kgroups[k] = (ntl[k] + e.nitems - 1) / e.nitems;
  e.item_base = 0;
  e.chunk_base = 0;
  e.n = n;
  e.eps = eps;
  e.b = b;
  e.x = x;
  if (o->record_history && o->history) {
    e.history = o->history;
    e.history_len = o->history_len;
  }
  if (o->lanczos && o->lanczos_len > 0) {
    e.lanczos = o->lanczos;
    e.lanczos_len = o->lanczos_len;
  }
  const int items = e.nitems, chunks = (e.nitems + kChunk - 1) / kChunk;
  const size_t off_sys = off; off += al(sizeof(EngSys));
  const size_t off_st0 = off; off += al(sizeof(EngState));
  const size_t off_st1 = off; off += al(sizeof(EngState));
  const size_t off_is = off; off += al(sizeof(int32_t) * items);
  const size_t off_it = off; off += al(sizeof(int32_t) * items);
  const size_t off_zero = off;  // everything from here to off_vec starts at zero
  const size_t off_part = off; off += al(sizeof(double) * 2 * items);
  const size_t off_cpart = off; off += al(sizeof(double) * 2 * chunks);
  const size_t off_cnt = off; off += al(sizeof(unsigned));
  const size_t off_ccnt = off; off += al(sizeof(unsigned) * chunks);
  const size_t off_gs = off; off += al(sizeof(GridSync));
  const int rgrid = 2 * num_sms();
  const size_t off_rpart = off; off += al(sizeof(double) * 2 * rgrid);
  const size_t off_vec = off;
  const size_t stride = al(n * sizeof(double));
  off += 7 * stride;
  if (off > kNoAllocBytes)
    return set_error(SPAI_ERR_TOO_LARGE, "allocation-free solve needs %zu bytes of scratch, %zu available", off,
                     kNoAllocBytes);
  unsigned char* vb = base + off_vec;
  e.r[0] = vb; e.r[1] = vb + stride;
  e.d[0] = vb + 2 * stride; e.d[1] = vb + 3 * stride;
  e.q = vb + 4 * stride; e.t = vb + 5 * stride; e.s = vb + 6 * stride;

  for (int k = 0; k < 3; ++k)
    if ((rc = launch_tiles(mats[k]->rowptr, n, mats[k]->nnz, tn, ntl[k],
                           reinterpret_cast<int32_t*>(base + off_tiles[k]), s)))
      return rc;
  EngState st;
  memset(&st, 0, sizeof(st));
  st.phase = PH_RESID0;
  st.status = SPAI_OK;
  std::vector<int32_t> isys(items, 0), itile(items);
  for (int v = 0; v < items; ++v) itile[v] = v;
  GridSync g0;
  memset(&g0, 0, sizeof(g0));
  g0.live = 1;
  g0.npos = items;  // item v at position v, no holes
  SPAI_CUDA(cudaMemsetAsync(base + off_zero, 0, off_vec - off_zero, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_sys, &e, sizeof(e), cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_st0, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_st1, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_is, isys.data(), sizeof(int32_t) * items, cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_it, itile.data(), sizeof(int32_t) * items, cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(base + off_gs, &g0, sizeof(g0), cudaMemcpyHostToDevice, s));

  EngArgs args;
  memset(&args, 0, sizeof(args));
  args.sys = reinterpret_cast<const EngSys*>(base + off_sys);
  args.st0 = reinterpret_cast<EngState*>(base + off_st0);
  args.st1 = reinterpret_cast<EngState*>(base + off_st1);
  args.nsys = 1;
  args.item_sys = reinterpret_cast<const int32_t*>(base + off_is);
  args.item_tile = reinterpret_cast<const int32_t*>(base + off_it);
  args.n_items = items;
  args.partial = reinterpret_cast<double*>(base + off_part);
  args.cpartial = reinterpret_cast<double*>(base + off_cpart);
  args.cnt = reinterpret_cast<unsigned*>(base + off_cnt);
  args.ccnt = reinterpret_cast<unsigned*>(base + off_ccnt);
  args.gs = reinterpret_cast<GridSync*>(base + off_gs);
  int64_t max_iter = o->max_iter;
  if (max_iter <= 0) max_iter = (10 * n < 1000000) ? 10 * n : 1000000;
  args.o.tol2 = o->rtol * o->rtol;
  args.o.reliable2 = 0.01;
  args.o.max_iter = max_iter;
  args.o.period = o->replace_period < 0 ? 0 : o->replace_period;
  args.o.criterion = o->criterion;
  args.o.max_outer = 0;
  args.o.mixed = 0;
  args.limit_ns = 2000000000ull;
  int grid = grid_max < items ? grid_max : items;
  if (grid < 1) grid = 1;
  const int64_t slot_cap = 8 * max_iter + 64;
  const int chunk = 3000;
  int64_t done_slots = 0;
  int launches = 0;
  for (;;) {
    const int64_t left = slot_cap - done_slots;
    args.max_slots = (int32_t)(left < chunk ? left : chunk);
    if (args.max_slots <= 0) break;
    void* kargs[] = {&args};
    SPAI_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(block), kargs, smem, s));
    count_launch();
    ++launches;
    GridSync gh;
    SPAI_CUDA(cudaMemcpyAsync(&gh, args.gs, sizeof(gh), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    done_slots = gh.slot;
    if (gh.err == kErrTable) return set_error(SPAI_ERR_INVALID, "engine: a launch-table entry was out of range");
    if (gh.err) return set_error(SPAI_ERR_TIMEOUT, "engine: a bounded device wait timed out");
    if (gh.live <= 0) break;
  }
  EngState fin;
  SPAI_CUDA(cudaMemcpyAsync(&fin, (done_slots & 1) ? args.st1 : args.st0, sizeof(fin), cudaMemcpyDeviceToHost, s));
  double* rpart = reinterpret_cast<double*>(base + off_rpart);
  true_residual_kernel<<<rgrid, 256, 0, s>>>(A->rowptr, A->colidx, static_cast<const double*>(A->val), b, x, n, rpart);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  std::vector<double> hp(2 * rgrid);
  SPAI_CUDA(cudaMemcpyAsync(hp.data(), rpart, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  double rr = 0, bb = 0;
  for (int k = 0; k < rgrid; ++k) { rr += hp[2 * k]; bb += hp[2 * k + 1]; }
  memset(res, 0, sizeof(*res));
  res->iters = fin.iter;
  res->outer_iters = 0;
  res->status = (fin.phase == PH_DONE) ? fin.status : SPAI_ERR_NOT_CONVERGED;
  res->true_rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
  res->rec_rel_res = fin.bb > 0 ? sqrt(fin.rr / fin.bb) : 0.0;
  res->history_written = fin.hist_n;
  if (e.lanczos) res->lanczos_written = fin.iter < e.lanczos_len ? fin.iter : e.lanczos_len;
  res->engine_ms = 0.0;
  res->slots = done_slots;
  res->launches = launches;
  if (res->status != SPAI_OK)
    set_error(res->status, "pcg: %s", res->status == SPAI_ERR_BREAKDOWN ? "breakdown" : "not converged");
  return res->status;
}
