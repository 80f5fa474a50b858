// Tensor-core (tcgen05) evaluation of the GNN's per-node MLP layers.
//
// A tile of 128 nodes is one MMA of M = 128 rows: D[128 x N] = X[128 x K] W^T,
// with X the node activations and W a layer's weights (N outputs, K inputs),
// both staged K-major in shared memory in the no-swizzle core-matrix layout
// (8 rows x 16 bytes per core matrix), D accumulated in tensor memory.
// Inputs are float32; each product is formed as three TF32 products
// (hi*hi + hi*lo + lo*hi, hi = x rounded to TF32, lo = the rounded rest), which
// keeps float32-level accuracy while running on the tensor pipe.
#pragma once

#include "internal.cuh"

namespace spai {
namespace tc {

constexpr int kM = 128;        // nodes per tile = MMA rows = TMEM lanes
constexpr int kKmax = 24;      // largest K (hidden width)
constexpr int kTmemCols = 128; // accumulator columns allocated (N <= 128)

// byte offset of element (row, k) in a K-major no-swizzle tile with K columns
__host__ __device__ __forceinline__ int core_off(int row, int k, int K) {
  return ((row >> 3) * (K >> 2) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;                // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  uint32_t d = 0;
  d |= 1u << 4;   // accumulate in F32
  d |= 2u << 7;   // A: TF32
  d |= 2u << 10;  // B: TF32
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(m >> 4) << 24;
  return d;       // both operands K-major
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One MMA of K = 8 (TF32): D (+)= A * B^T.
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 accumulator columns of this thread's TMEM lane (row).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Issued by one thread: D[128 x N] = A * B^T over K (multiple of 8) with the
// three split products; A_hi/A_lo, B_hi/B_lo K-major no-swizzle tiles.
__device__ __forceinline__ void gemm3(uint32_t tmem_d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                      int K, int N) {
  const uint32_t idesc = idesc_tf32(kM, N);
  const uint32_t lbo = 128, sbo = (uint32_t)(K >> 2) * 128;
  uint32_t acc = 0;
  for (int term = 0; term < 3; ++term) {
    const uint32_t a = term == 2 ? a_lo : a_hi;
    const uint32_t b = term == 1 ? b_lo : b_hi;
    for (int ks = 0; ks < K / 8; ++ks) {
      mma_tf32(tmem_d, smem_desc(a + ks * 256, lbo, sbo), smem_desc(b + ks * 256, lbo, sbo), idesc, acc);
      acc = 1;
    }
  }
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, unsigned parity, uint64_t limit_ns) {
  return mbar_wait_bounded(bar, parity, limit_ns);
}
#endif  // __CUDACC__

}  // namespace tc
}  // namespace spai
