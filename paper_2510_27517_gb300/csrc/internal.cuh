// Internal definitions shared by the library's translation units.
// Nothing here is part of the public ABI (see include/spai.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "spai.h"

namespace spai {

// ---------------------------------------------------------------------------
// Host-side error state
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
void count_launch(int n = 1);
int cuda_error(cudaError_t e, const char* what);

#define SPAI_CUDA(call)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::spai::cuda_error(_e, #call); \
  } while (0)

// Device allocation tied to a stream (stream-ordered pool allocator).
// Temporaries are freed stream-ordered on the stream they were allocated on;
// memory owned by a handle (keep() called) is freed with cudaFree, which
// waits for all work, because the creating stream may be gone by then.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  bool owned = false;
  void keep() { owned = true; }
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  int alloc(size_t nbytes, cudaStream_t stream);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

size_t dtype_size(int dt);

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
// SELL-32 layout of a CSR pattern: slices of 32 rows, each slice stored
// column-major (entry k of the slice's 32 rows together) with the width of
// its longest row.  Entry k of the row at slice position p (slice p / 32,
// lane p % 32) sits at sptr[p / 32] + 32 k + p % 32; positions past a row's
// length are padding (column 0, value 0).  Plain SELL-32 keeps row i at
// position i.  Where that pads more than a quarter (irregular rows), the
// rows of every window of kSellSigma consecutive rows are ordered by
// decreasing length (SELL-C-sigma; stable, so equal lengths keep their
// order) and rows[p] holds the row at position p (n for the padding lanes
// past the last row).  Built only when every row has at most kSellMaxRow
// entries and the padding adds at most a quarter to the stored entries.
constexpr int32_t kSellMaxRow = 64;
constexpr int32_t kSellSigma = 1024;
struct SellData {
  int32_t nslices = 0;         // 0: not available
  int32_t max_width = 0;
  int32_t block = 1;           // 3: the 3 x 3 block layout of bsell.cu (entries and widths count blocks)
  int64_t total = 0;           // stored entries including padding
  DevMem sptr;                 // nslices + 1 entry offsets (multiples of 32)
  DevMem ci;                   // total column indices
  DevMem rows;                 // 32 nslices row indices (sorted layout only; empty: row = position)
  const int32_t* row_map() const { return rows.as<int32_t>(); }
};

struct PatternData {
  int64_t n = 0, nnz = 0;      // nnz of G
  int32_t kind = SPAI_PATTERN_FULL;
  int32_t max_row = 0;         // longest row of G
  int32_t max_row_t = 0;       // longest row of G^T
  DevMem rowptr, colidx;       // G
  DevMem t_rowptr, t_colidx;   // G^T (separate arrays for LOWER/UPPER; empty for FULL)
  DevMem perm;                 // val_T[perm[e]] = val[e]
  DevMem src;                  // index into A of each entry of G (LOWER/UPPER only)
  int64_t a_nnz = 0;           // nnz of the A it was built from
  SellData sell;               // FULL patterns (shared by G and G^T)
  SellData bsell;              // FULL patterns made of dense 3 x 3 blocks
  const int32_t* g_rp() const { return rowptr.as<int32_t>(); }
  const int32_t* g_ci() const { return colidx.as<int32_t>(); }
  const int32_t* gt_rp() const { return kind == SPAI_PATTERN_FULL ? rowptr.as<int32_t>() : t_rowptr.as<int32_t>(); }
  const int32_t* gt_ci() const { return kind == SPAI_PATTERN_FULL ? colidx.as<int32_t>() : t_colidx.as<int32_t>(); }
};

// Row-start table of one matrix for one tile size (built on demand, cached
// for the last (offset array, tile size) pair).
struct TileSet {
  int32_t tile_nnz = 0;
  int32_t ntiles = 0;
  const void* src = nullptr;
  DevMem starts;  // ntiles + 1 row (or slice) indices
};


struct PrecondData {
  std::shared_ptr<PatternData> P;
  int32_t gtype = SPAI_F64;
  double eps = 0.0;
  double anorm = 0.0;        // ||A|| used by the GNN (0 when values were given)
  DevMem g_val, gt_val;
  DevMem sell_g, sell_gt;    // values in the pattern's SELL-32 layout (when it has one)
  DevMem bsell_g, bsell_gt;  // values in the pattern's 3 x 3 block layout (when it has one)
  TileSet g_tiles, gt_tiles; // cached for the last tile size used
};

struct SystemData {
  int64_t n = 0, nnz = 0;
  int32_t max_row = 0;
  DevMem rowptr, colidx, val64, val32;
  // SpMV schedule of the persistent solver (the same for A, G^T and G):
  int32_t tile_nnz = 2048;   // entries per row group (one staging unit)
  int32_t items_log2 = 0;    // groups per work item = heuristic count * 2^items_log2
  int32_t staged = 1;        // 1: groups staged by TMA bulk copies (when rows fit), 0: direct loads
  int32_t sell = 1;          // 1: SELL-32 layout for matrices that have one, 0: CSR row groups
  int32_t fuse = 1;          // 1: G^T and G passes in one grid step ordered by item flags
  int32_t block = 1;         // 1: the 3 x 3 block layout for matrices that have it (A and G)
  int32_t pair = 0;          // 1: s with d and q with r stored as interleaved pairs (set for sorted rows)
  int32_t autotune = 0;      // pick the schedule by timing candidates on the first solve
  int32_t tuned = 0;
  TileSet tiles;
  SellData sell_a;           // A in SELL-32 (pattern and float64 / float32 values)
  DevMem sell_v64, sell_v32;
  SellData bsell_a;          // A in the 3 x 3 block layout (when it is made of dense 3 x 3 blocks)
  DevMem bsell_v64, bsell_v32;
};

}  // namespace spai

struct spai_pattern { std::shared_ptr<spai::PatternData> d; };
struct spai_precond { std::shared_ptr<spai::PrecondData> d; };
struct spai_system  { std::shared_ptr<spai::SystemData> d; };

namespace spai {

// Internal entry points used across translation units.
int build_tiles(const int32_t* rowptr, int64_t n, int64_t nnz, int32_t tile_nnz, TileSet& ts, cudaStream_t s);
int validate_csr_device(const spai_csr* A, bool need_symmetric, int32_t* max_row, cudaStream_t s);
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
int system_from_csr(const spai_csr* A, SystemData& S, bool validate, cudaStream_t s);
// SELL-32 pattern of a CSR (out.nslices stays 0 when the layout does not pay)
int build_sell(const int32_t* rp, const int32_t* ci, int64_t n, int64_t nnz, int32_t max_row, SellData& out,
               cudaStream_t s);
// values of a CSR (dtype dt_in) into the SELL-32 layout (dtype dt_out)
int sell_values(const SellData& L, const int32_t* rp, int64_t n, const void* val, int dt_in, void* out, int dt_out,
                cudaStream_t s);
// G and G^T values of a preconditioner in its pattern's SELL-32 and 3 x 3 block layouts
int precond_sell(PrecondData& M, cudaStream_t s);
// 3 x 3 block layout of a CSR made of dense 3 x 3 blocks (out.nslices stays 0 otherwise)
int build_bsell(const int32_t* rp, const int32_t* ci, int64_t n, int64_t nnz, SellData& out, cudaStream_t s);
// values of such a CSR (dtype dt_in) into the block layout (dtype dt_out, 9 per block)
int bsell_values(const SellData& L, const int32_t* rp, int64_t n, const void* val, int dt_in, void* out, int dt_out,
                 cudaStream_t s);
// ||A|| = mean |A_ij| (Sec. 3.3) into out[0] (device), deterministic
int matrix_abs_mean(const double* val, int64_t nnz, double* out, cudaStream_t s);
int num_sms();

// Bytes of engine workspace of one system (its iteration vectors); `pair`:
// the interleaved layout of s with d and q with r (two vectors longer).
size_t engine_work_bytes(int64_t n, bool mixed, bool pair);

// Session interface of the engine, used by the server: a batch whose members
// carry their state (an opaque block of engine_state_bytes()) across launches.
struct SessionMember {
  SystemData* S;
  PrecondData* M;
  const double* b;
  double* x;
  void* work;                        // engine_work_bytes(S->n, mixed, pair) bytes
  int32_t pair;                      // the vector layout `work` was sized and started for
  std::vector<unsigned char> state;  // empty: start a new solve
};
struct SessionView {
  bool done;
  int status;
  int64_t iters;
  int outer;
};
struct EngineSession;
size_t engine_state_bytes();
int session_create(bool mixed, int gtype, const spai_pcg_opts& o, cudaStream_t s, EngineSession** out);
int session_set(EngineSession* es, std::vector<SessionMember>& members);
int session_launch(EngineSession* es, int max_slots);
int session_live(EngineSession* es);
int session_read(EngineSession* es, std::vector<SessionMember>& members, std::vector<SessionView>& views);
void session_destroy(EngineSession* es);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Loads of vectors written by other blocks before the last grid barrier
// (ordinary cached loads; the barrier's fences order them).
template <class T> __device__ __forceinline__ T ldv(const T* p) { return *p; }

// Loads of data written earlier in the same kernel by other blocks without an
// intervening grid barrier (reduction partials, states): bypass L1.
template <class T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ldcg(const __nv_bfloat16* p) {
  unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(p));
  return __ushort_as_bfloat16(u);
}
template <> __device__ __forceinline__ __half ldcg(const __half* p) {
  unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(p));
  return __ushort_as_half(u);
}

// Read-only streams (matrix data): read-only path.
template <class T> __device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ double to_f64(__half v) { return (double)__half2float(v); }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

// Separately rounded arithmetic (no contraction into FMA), so that vector
// updates round exactly like  a + b * c  evaluated as two operations.
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
// a * b + c with one rounding
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed shuffle tree, then fixed order over warps).
// `scratch` needs blockDim.x/32 doubles.  Result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  __syncthreads();
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// ---- TMA bulk copies (global -> shared) completing on an mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  uint64_t st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(st) : "r"(smem_u32(bar)), "r"(bytes) : "memory");
  (void)st;
}
// L2 policy for data streamed once (matrix entries): evicted first, so the
// vectors gathered by the SpMVs stay resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_1d_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; false if `limit_ns` passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Two deterministic block sums in one pass; `scratch` needs 2 * warps doubles.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* scratch) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    scratch[w] = a;
    scratch[nw + w] = b;
  }
  __syncthreads();
  if (w == 0) {
    double ta = (l < nw) ? scratch[l] : 0.0;
    double tb = (l < nw) ? scratch[nw + l] : 0.0;
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    if (l == 0) {
      scratch[0] = ta;
      scratch[nw] = tb;
    }
  }
  __syncthreads();
  a = scratch[0];
  b = scratch[nw];
  __syncthreads();
}

// Grid-wide barrier for cooperative launches with a bounded wait.  (A
// two-level arrival count -- per-group counters, then a counter of groups --
// measured slower on GB300 than one counter: the last arriver's chain of two
// atomics outweighs the serialised arrivals.)
struct GridSync {
  unsigned count;  // blocks arrived
  unsigned gen;    // generation (counts in steps of 2); bit 0: the exit decided at the last barrier
  int npos;        // positions of the launch table in use (holes included)
  int err;         // SPAI_ERR_TIMEOUT when a wait gave up
  int live;        // systems still running
  int slot;        // slots executed so far (parity of double-buffered state)
  int pad[2];
};

// Returns the exit flag decided at this barrier.  Every wait is bounded by
// `limit_ns`; on expiry err is set and the caller must stop.  Arrival is an
// acq_rel atomic (releases this block's writes, and the last arriver acquires
// everyone's); the last arriver publishes the next generation with a release
// store and the others acquire it, so writes made before the barrier by any
// block are visible after it (the CTA barrier extends this to every thread).
// The exit decision (no live system, or an error) travels in bit 0 of the
// generation word, so a waiter needs no further load after its wait.
__device__ __forceinline__ int grid_barrier(GridSync* g, unsigned nblocks, uint64_t limit_ns, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned my_gen = ld_relaxed_u32(&g->gen);
    const unsigned prev = atom_add_acq_rel_u32(&g->count, 1u);
    unsigned ex;
    if (prev == nblocks - 1) {
      g->count = 0;
      const int live = *(volatile int*)&g->live;
      const int err = *(volatile int*)&g->err;
      ex = (live <= 0 || err != 0) ? 1u : 0u;
      st_release_u32(&g->gen, ((my_gen | 1u) + 1u) | ex);
    } else {
      const uint64_t t0 = global_ns();
      unsigned spins = 0, v;
      bool gave_up = false;
      while ((v = ld_acquire_u32(&g->gen)) == my_gen) {
        if ((++spins & 1023u) == 0 && global_ns() - t0 > limit_ns) {
          atomicExch(&g->err, SPAI_ERR_TIMEOUT);
          gave_up = true;
          break;
        }
      }
      ex = gave_up ? 1u : (v & 1u);
    }
    *sflag = (int)ex;
  }
  __syncthreads();
  return *sflag;
}

// ---- item flags: ordering of the two passes of a fused grid step ----
// A G-pass item may start gathering t once every G^T-pass item whose rows it
// reaches has published the current step's epoch.  Warp 0 polls the flags
// with relaxed loads (an acquire per poll would invalidate L1 for the other
// blocks of the SM), then one acquire fence makes the producers' writes
// visible and the block barrier extends that to every thread.  Bounded: on
// expiry the error flag is set and the step's results are dropped.
struct ItemWait {
  const unsigned* f;  // nullptr: no wait
  int lo, hi;         // inclusive item range
  unsigned epoch;
};

static __device__ __noinline__ void wait_items(const ItemWait W, uint64_t limit_ns, int* err) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint64_t t0 = 0;
    unsigned spins = 0;
    bool expired = false;
    for (int u0 = W.lo; u0 <= W.hi && !expired; u0 += 32) {
      const int u = u0 + lane;
      bool ready = u > W.hi || (int)(ld_relaxed_u32(W.f + u) - W.epoch) >= 0;
      while (!__all_sync(0xffffffffu, ready)) {
        if (!ready) ready = (int)(ld_relaxed_u32(W.f + u) - W.epoch) >= 0;
        if ((++spins & 255u) == 0) {
          int ex = 0;
          if (lane == 0) {
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) ex = 1;
          }
          if (__shfl_sync(0xffffffffu, ex, 0)) {
            if (lane == 0) atomicExch(err, SPAI_ERR_TIMEOUT);
            expired = true;
            break;
          }
        }
      }
    }
    if (lane == 0) fence_acq_rel_gpu();
  }
  __syncthreads();
}

#endif  // __CUDACC__

}  // namespace spai
