// 3 x 3 block layout of a CSR matrix made of dense 3 x 3 blocks (Sec. 3.2.2
// writes G in b x b blocks for systems with three unknowns per node, the
// paper's hyperelastic workload): slices of 32 block rows stored
// column-major with one column index per block.  A block row I (scalar rows
// 3I .. 3I + 2) qualifies when its three scalar rows list the same blocks in
// column order, three consecutive columns 3J, 3J + 1, 3J + 2 per block.
//
// Layout (SellData with block = 3): slice s holds block rows 32 s .. 32 s + 31
// and has the width w_s of its longest block row; sptr[s] counts blocks
// (a multiple of 32); block q of the block row at lane l has its block
// column J at ci[sptr[s] + 32 q + l] and its value (r, c) at
// val[9 sptr[s] + 32 (9 q + 3 r + c) + l] -- every (q, r, c) position is one
// coalesced warp load.  Padding blocks: column 0, values 0.
#include <algorithm>

#include "internal.cuh"

namespace spai {
namespace {

int grid_of(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// One thread per block row: its block count, or a flag if the rows are not
// made of aligned dense 3 x 3 blocks.
__global__ void bsell_count_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nb,
                                   int32_t* __restrict__ nblk, int* bad) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nb; I += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = 3 * I;
    const int len = rp[r0 + 1] - rp[r0];
    bool ok = len % 3 == 0;
    for (int r = 1; ok && r < 3; ++r) ok = rp[r0 + r + 1] - rp[r0 + r] == len;
    for (int q = 0; ok && q < len / 3; ++q) {
      const int32_t j0 = ci[rp[r0] + 3 * q];
      ok = j0 % 3 == 0;
      for (int r = 0; ok && r < 3; ++r)
        for (int c = 0; ok && c < 3; ++c) ok = ci[rp[r0 + r] + 3 * q + c] == j0 + c;
    }
    nblk[I] = ok ? len / 3 : 0;
    if (!ok) atomicOr(bad, 1);
  }
}

// 32 x (most blocks in a block row) of every slice; one warp per slice
__global__ void bsell_width_kernel(const int32_t* __restrict__ nblk, int64_t nb, int64_t nslices, int32_t* w32) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nw) {
    const int64_t I = sl * 32 + lane;
    int w = I < nb ? nblk[I] : 0;
    for (int o = 16; o; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (lane == 0) w32[sl] = 32 * w;
  }
}

__device__ __forceinline__ double ld_any(const void* p, int dt, int64_t i) {
  switch (dt) {
    case SPAI_F64: return static_cast<const double*>(p)[i];
    case SPAI_F32: return (double)static_cast<const float*>(p)[i];
    case SPAI_BF16: return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    default: return (double)__half2float(static_cast<const __half*>(p)[i]);
  }
}

__device__ __forceinline__ void st_any(void* p, int dt, int64_t i, double v) {
  switch (dt) {
    case SPAI_F64: static_cast<double*>(p)[i] = v; break;
    case SPAI_F32: static_cast<float*>(p)[i] = (float)v; break;
    case SPAI_BF16: static_cast<__nv_bfloat16*>(p)[i] = __double2bfloat16(v); break;
    default: static_cast<__half*>(p)[i] = __double2half(v); break;
  }
}

// One thread per block position (32 nslices): the block columns (when ci_out
// is given) and the 9 values of every block (when val_out is given).
__global__ void bsell_fill_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t nb,
                                  int64_t nslices, const int32_t* __restrict__ sptr, int32_t* ci_out,
                                  const void* val, int dt_in, void* val_out, int dt_out) {
  const int64_t npos = nslices * 32;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = p >> 5;
    const int lane = (int)(p & 31);
    const int64_t off = sptr[sl];
    const int w = (sptr[sl + 1] - sptr[sl]) >> 5;
    const int64_t I = p;
    const int nbl = I < nb ? (rp[3 * I + 1] - rp[3 * I]) / 3 : 0;
    for (int q = 0; q < w; ++q) {
      const bool real = q < nbl;
      if (ci_out) ci_out[off + 32 * (int64_t)q + lane] = real ? ci[rp[3 * I] + 3 * q] / 3 : 0;
      if (val_out)
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            st_any(val_out, dt_out, 9 * off + 32 * (int64_t)(9 * q + 3 * r + c) + lane,
                   real ? ld_any(val, dt_in, rp[3 * I + r] + 3 * q + c) : 0.0);
    }
  }
}

}  // namespace

int build_bsell(const int32_t* rp, const int32_t* ci, int64_t n, int64_t nnz, SellData& out, cudaStream_t s) {
  out.nslices = 0;
  out.total = 0;
  out.block = 3;
  if (n <= 0 || n % 3 != 0 || nnz % 9 != 0) return SPAI_OK;
  const int64_t nb = n / 3;
  const int64_t ns = (nb + 31) / 32;
  int rc;
  DevMem nblk, w, flag;
  if ((rc = nblk.alloc((size_t)nb * sizeof(int32_t), s))) return rc;
  if ((rc = w.alloc((size_t)(ns + 1) * sizeof(int32_t), s))) return rc;
  if ((rc = flag.alloc(sizeof(int), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  bsell_count_kernel<<<grid_of(nb, 256), 256, 0, s>>>(rp, ci, nb, nblk.as<int32_t>(), flag.as<int>());
  count_launch();
  SPAI_CUDA(cudaMemsetAsync(w.as<int32_t>() + ns, 0, sizeof(int32_t), s));
  bsell_width_kernel<<<grid_of(ns * 32, 256), 256, 0, s>>>(nblk.as<int32_t>(), nb, ns, w.as<int32_t>());
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  DevMem& sptr = out.sptr;
  if ((rc = sptr.alloc((ns + 1 + 16) * sizeof(int32_t), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(sptr.p, 0, (ns + 1 + 16) * sizeof(int32_t), s));
  if ((rc = exclusive_scan_i32(w.as<int32_t>(), sptr.as<int32_t>(), ns + 1, s))) return rc;
  int32_t total = 0, bad = 0;
  SPAI_CUDA(cudaMemcpyAsync(&total, sptr.as<int32_t>() + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  // not made of 3 x 3 blocks, or padding would add more than a quarter
  if (bad || (int64_t)total * 9 * 4 > nnz * 5 || (int64_t)total * 9 >= (int64_t)INT32_MAX - 1024) {
    sptr.release();
    return SPAI_OK;
  }
  const int64_t pad = 64;
  if ((rc = out.ci.alloc((total + pad) * sizeof(int32_t), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(out.ci.p, 0, (total + pad) * sizeof(int32_t), s));
  bsell_fill_kernel<<<grid_of(ns * 32, 256), 256, 0, s>>>(rp, ci, nb, ns, sptr.as<int32_t>(), out.ci.as<int32_t>(),
                                                           nullptr, 0, nullptr, 0);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  out.sptr.keep();
  out.ci.keep();
  out.nslices = (int32_t)ns;
  out.total = total;
  int32_t mw = 0;
  {
    std::vector<int32_t> hs(ns + 1);
    SPAI_CUDA(cudaMemcpyAsync(hs.data(), sptr.p, (ns + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < ns; ++i) mw = std::max(mw, (hs[i + 1] - hs[i]) / 32);
  }
  out.max_width = mw;
  return SPAI_OK;
}

// Values (9 per stored block, zeros in padding) of a block-structured CSR in
// the layout L, converted from dt_in to dt_out; `out` holds 9 L.total values.
int bsell_values(const SellData& L, const int32_t* rp, int64_t n, const void* val, int dt_in, void* out, int dt_out,
                 cudaStream_t s) {
  if (L.nslices <= 0 || L.block != 3) return set_error(SPAI_ERR_INVALID, "no 3 x 3 block layout");
  bsell_fill_kernel<<<grid_of((int64_t)L.nslices * 32, 256), 256, 0, s>>>(rp, nullptr, n / 3, L.nslices,
                                                                           L.sptr.as<int32_t>(), nullptr, val, dt_in,
                                                                           out, dt_out);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

}  // namespace spai
