// Sparsity pattern of G and its explicit transpose (build_pattern), CSR
// validation, scans and SpMV tile tables.
//
// Sec. 3.2.2 (after Eq. 5): G is written on A's sparsity pattern.  Storing
// G^T as its own CSR makes both products of the apply s = G (G^T r) + eps r
// (Eq. 1, Eq. 2) row gathers, so no kernel needs atomics.  Because A is SPD
// its pattern is symmetric, so the transpose of a pattern restricted to one
// triangle is the restriction to the other triangle, and the position of the
// mirror entry (j, i) is found by a binary search in row j.  Every output is
// a pure function of the input pattern (bit-exact, no atomics on the data).
#include <cstdio>

#include "internal.cuh"

namespace spai {

namespace {

constexpr int kBadRowptr = 1, kBadCol = 2, kUnsorted = 4, kNoDiag = 8, kAsym = 16, kTooBig = 32;

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int lo, int hi, int key) {
  // first position p in [lo, hi) with a[p] >= key (hi if none)
  while (lo < hi) {
    int mid = lo + ((hi - lo) >> 1);
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One warp per row.  Checks rowptr monotonicity, column range, strictly
// ascending columns, the diagonal and (optionally) the mirror entry.
__global__ void validate_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                                int64_t nnz, int check_sym, int* flags, int* max_row) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const int b = __ldg(rp + i), e = __ldg(rp + i + 1);
    if (b < 0 || e < b || e > nnz) {
      if (lane == 0) atomicOr(flags, kBadRowptr);
      continue;
    }
    if (lane == 0) atomicMax(max_row, e - b);
    bool diag = false;
    int bad = 0;
    for (int k = b + lane; k < e; k += 32) {
      const int c = __ldg(ci + k);
      if (c < 0 || c >= n) { bad |= kBadCol; continue; }
      if (k > b && __ldg(ci + k - 1) >= c) bad |= kUnsorted;
      if (c == i) diag = true;
      if (check_sym && c != i) {
        const int cb = __ldg(rp + c), ce = __ldg(rp + c + 1);
        if (cb < 0 || ce < cb || ce > nnz) { bad |= kBadRowptr; continue; }
        const int p = lower_bound_i32(ci, cb, ce, (int)i);
        if (p >= ce || __ldg(ci + p) != i) bad |= kAsym;
      }
    }
    const unsigned any_diag = __ballot_sync(0xffffffffu, diag);
    if (bad) atomicOr(flags, bad);
    if (lane == 0 && !any_diag) atomicOr(flags, kNoDiag);
  }
}

__global__ void check_ends_kernel(const int32_t* rp, int64_t n, int64_t nnz, int* flags) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (rp[0] != 0 || (int64_t)rp[n] != nnz) atomicOr(flags, kBadRowptr);
  }
}

// ----- scan -----
constexpr int kScanBlock = 1024;

__global__ void scan_block_kernel(const int32_t* in, int32_t* out, int32_t* block_sums, int64_t n) {
  __shared__ int32_t s[kScanBlock];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int32_t v = (i < n) ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    int32_t t = (threadIdx.x >= o) ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == kScanBlock - 1 && block_sums) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_add_kernel(int32_t* out, const int32_t* offs, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

// ----- pattern construction -----
__global__ void count_tri_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                                 int lower, int32_t* counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = rp[i], e = rp[i + 1];
    // columns ascending: count of c <= i (lower) or c >= i (upper) by search
    int p = b;
    {
      int lo = b, hi = e;
      const int key = lower ? (int)i + 1 : (int)i;
      while (lo < hi) { int m = lo + ((hi - lo) >> 1); if (ci[m] < key) lo = m + 1; else hi = m; }
      p = lo;
    }
    counts[i] = lower ? (p - b) : (e - p);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) counts[n] = 0;
}

__global__ void compact_tri_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                                   int lower, const int32_t* __restrict__ out_rp, int32_t* out_ci, int32_t* src) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = rp[i], e = rp[i + 1];
    int o = out_rp[i];
    for (int k = b; k < e; ++k) {
      const int c = ci[k];
      if (lower ? (c <= i) : (c >= i)) {
        out_ci[o] = c;
        if (src) src[o] = k;
        ++o;
      }
    }
  }
}

// perm[e] = position of the mirror entry (col(e), row(e)) in the transposed CSR.
__global__ void perm_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const int32_t* __restrict__ t_rp, const int32_t* __restrict__ t_ci, int64_t n,
                            int32_t* perm, int* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = rp[i], e = rp[i + 1];
    for (int k = b; k < e; ++k) {
      const int j = ci[k];
      const int p = lower_bound_i32(t_ci, t_rp[j], t_rp[j + 1], (int)i);
      if (p >= t_rp[j + 1] || t_ci[p] != i) { atomicOr(flags, kAsym); perm[k] = 0; }
      else perm[k] = p;
    }
  }
}

__global__ void tiles_kernel(const int32_t* __restrict__ rp, int64_t n, int64_t nnz, int32_t tile_nnz,
                             int32_t ntiles, int32_t* starts) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= ntiles; j += (int64_t)gridDim.x * blockDim.x) {
    if (j == ntiles) { starts[j] = (int32_t)n; continue; }
    const int64_t key = j * (int64_t)tile_nnz;
    int64_t lo = 0, hi = n;  // first row whose start offset >= key
    while (lo < hi) { int64_t m = lo + ((hi - lo) >> 1); if ((int64_t)rp[m] < key) lo = m + 1; else hi = m; }
    starts[j] = (int32_t)lo;
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

std::string flag_text(int f) {
  std::string s;
  if (f & kBadRowptr) s += "rowptr not monotone / out of range; ";
  if (f & kBadCol) s += "column index out of range; ";
  if (f & kUnsorted) s += "columns not strictly ascending; ";
  if (f & kNoDiag) s += "missing diagonal; ";
  if (f & kAsym) s += "pattern not symmetric; ";
  if (f & kTooBig) s += "too large; ";
  return s;
}

}  // namespace

// Launchers over caller-provided memory (no allocation): CSR validation into
// flags[0] (defect bits) and flags[1] (longest row), and the tile table.
int launch_validate(const spai_csr* A, int check_sym, int* flags, cudaStream_t s) {
  check_ends_kernel<<<1, 32, 0, s>>>(A->rowptr, A->n, A->nnz, flags); count_launch();
  SPAI_CUDA(cudaGetLastError());
  if (A->n > 0) {
    validate_kernel<<<grid_for(A->n * 32, 256), 256, 0, s>>>(A->rowptr, A->colidx, A->n, A->nnz, check_sym, flags,
                                                             flags + 1); count_launch();
    SPAI_CUDA(cudaGetLastError());
  }
  return SPAI_OK;
}

std::string validate_flag_text(int f) { return flag_text(f); }

int launch_tiles(const int32_t* rowptr, int64_t n, int64_t nnz, int32_t tile_nnz, int32_t ntiles, int32_t* starts,
                 cudaStream_t s) {
  tiles_kernel<<<grid_for(ntiles + 1, 256), 256, 0, s>>>(rowptr, n, nnz, tile_nnz, ntiles, starts); count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return SPAI_OK;
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb == 1) {
    scan_block_kernel<<<1, kScanBlock, 0, s>>>(in, out, nullptr, n); count_launch();
    SPAI_CUDA(cudaGetLastError());
    return SPAI_OK;
  }
  DevMem sums, offs;
  int rc;
  if ((rc = sums.alloc(nb * sizeof(int32_t), s))) return rc;
  if ((rc = offs.alloc(nb * sizeof(int32_t), s))) return rc;
  scan_block_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, sums.as<int32_t>(), n); count_launch();
  SPAI_CUDA(cudaGetLastError());
  if ((rc = exclusive_scan_i32(sums.as<int32_t>(), offs.as<int32_t>(), nb, s))) return rc;
  scan_add_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(out, offs.as<int32_t>(), n); count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

int validate_csr_device(const spai_csr* A, bool need_symmetric, int32_t* max_row, cudaStream_t s) {
  if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->rowptr || (A->nnz > 0 && !A->colidx))))
    return set_error(SPAI_ERR_INVALID, "invalid CSR descriptor");
  if (A->n >= INT32_MAX || A->nnz >= INT32_MAX)
    return set_error(SPAI_ERR_BAD_CSR, "n or nnz exceeds int32 range");
  DevMem fl;
  int rc;
  if ((rc = fl.alloc(2 * sizeof(int), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(fl.p, 0, 2 * sizeof(int), s));
  int* flags = fl.as<int>();
  check_ends_kernel<<<1, 32, 0, s>>>(A->rowptr, A->n, A->nnz, flags); count_launch();
  SPAI_CUDA(cudaGetLastError());
  if (A->n > 0) {
    const int block = 256;
    const int64_t warps = A->n;
    int grid = grid_for(warps * 32, block);
    validate_kernel<<<grid, block, 0, s>>>(A->rowptr, A->colidx, A->n, A->nnz, need_symmetric ? 1 : 0, flags,
                                          flags + 1); count_launch();
    SPAI_CUDA(cudaGetLastError());
  }
  int h[2] = {0, 0};
  SPAI_CUDA(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  if (h[0]) return set_error(SPAI_ERR_BAD_CSR, "invalid CSR: %s", flag_text(h[0]).c_str());
  if (max_row) *max_row = h[1];
  return SPAI_OK;
}

int build_tiles(const int32_t* rowptr, int64_t n, int64_t nnz, int32_t tile_nnz, TileSet& ts, cudaStream_t s) {
  if (tile_nnz <= 0) return set_error(SPAI_ERR_INVALID, "tile size must be positive");
  if (ts.tile_nnz == tile_nnz && ts.src == rowptr && ts.starts.p) return SPAI_OK;
  int64_t nt = (nnz + tile_nnz - 1) / tile_nnz;
  if (nt < 1) nt = 1;
  if (nt >= INT32_MAX) return set_error(SPAI_ERR_INVALID, "too many tiles");
  int rc;
  ts.starts.release();
  if ((rc = ts.starts.alloc((nt + 1) * sizeof(int32_t), s))) return rc;
  tiles_kernel<<<grid_for(nt + 1, 256), 256, 0, s>>>(rowptr, n, nnz, tile_nnz, (int32_t)nt, ts.starts.as<int32_t>()); count_launch();
  SPAI_CUDA(cudaGetLastError());
  ts.starts.keep();
  ts.ntiles = (int32_t)nt;
  ts.tile_nnz = tile_nnz;
  ts.src = rowptr;
  return SPAI_OK;
}

int system_from_csr(const spai_csr* A, SystemData& S, bool validate, cudaStream_t s) {
  if (!A) return set_error(SPAI_ERR_INVALID, "A is NULL");
  if (A->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A values must be SPAI_F64");
  if (A->n <= 0) return set_error(SPAI_ERR_INVALID, "A must have n > 0");
  int rc;
  int32_t mr = 0;
  if (validate) {
    if ((rc = validate_csr_device(A, false, &mr, s))) return rc;
  } else {
    mr = 0;
  }
  S.n = A->n;
  S.nnz = A->nnz;
  S.max_row = mr;
  const int64_t pad = 16;
  if ((rc = S.rowptr.alloc((A->n + 1 + pad) * sizeof(int32_t), s))) return rc;
  if ((rc = S.colidx.alloc((A->nnz + pad) * sizeof(int32_t), s))) return rc;
  if ((rc = S.val64.alloc((A->nnz + pad) * sizeof(double), s))) return rc;
  if ((rc = S.val32.alloc((A->nnz + pad) * sizeof(float), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(S.colidx.p, 0, (A->nnz + pad) * sizeof(int32_t), s));
  SPAI_CUDA(cudaMemcpyAsync(S.rowptr.p, A->rowptr, (A->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(S.colidx.p, A->colidx, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(S.val64.p, A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  f64_to_f32_kernel<<<grid_for(A->nnz, 256), 256, 0, s>>>(S.val64.as<double>(), S.val32.as<float>(), A->nnz); count_launch();
  SPAI_CUDA(cudaGetLastError());
  S.tiles.starts.release();
  S.tiles.ntiles = 0;
  S.tiles.tile_nnz = 0;
  return SPAI_OK;
}

namespace {
// Row at SELL position p: p itself, or the sorted layout's row map.
__device__ __forceinline__ int64_t sell_row(const int32_t* __restrict__ rows, int64_t p) {
  return rows ? (int64_t)rows[p] : p;
}

// 32 x (longest row) of every 32-row slice; one warp per slice
__global__ void sell_width_kernel(const int32_t* __restrict__ rp, int64_t n, int64_t nslices, int32_t* w32,
                                  const int32_t* __restrict__ rows) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nw) {
    const int64_t row = sell_row(rows, sl * 32 + lane);
    int len = row < n ? rp[row + 1] - rp[row] : 0;
    for (int o = 16; o; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) w32[sl] = 32 * len;
  }
}

__device__ __forceinline__ double ld_dt(const void* p, int dt, int64_t i) {
  switch (dt) {
    case SPAI_F64: return static_cast<const double*>(p)[i];
    case SPAI_F32: return (double)static_cast<const float*>(p)[i];
    case SPAI_BF16: return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    default: return (double)__half2float(static_cast<const __half*>(p)[i]);
  }
}

// Stores v (exactly representable in dt whenever it came from dt or from a
// float64 value rounded once to dt) at index i of an array of type dt.
__device__ __forceinline__ void st_dt(void* p, int dt, int64_t i, double v) {
  switch (dt) {
    case SPAI_F64: static_cast<double*>(p)[i] = v; break;
    case SPAI_F32: static_cast<float*>(p)[i] = (float)v; break;
    case SPAI_BF16: static_cast<__nv_bfloat16*>(p)[i] = __double2bfloat16(v); break;
    default: static_cast<__half*>(p)[i] = __double2half(v); break;
  }
}

// Row windows of kSellSigma rows, one thread each: the positions of the
// window's rows ordered by decreasing length, rows of equal length in row
// order (a stable counting sort over lengths 0..kSellMaxRow); positions past
// the last row get n.
__global__ void sell_sort_kernel(const int32_t* __restrict__ rp, int64_t n, int64_t npos, int32_t* __restrict__ rows) {
  const int64_t nwin = (npos + kSellSigma - 1) / kSellSigma;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwin; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = w * kSellSigma;
    const int64_t r1 = min(r0 + kSellSigma, n);
    int cnt[kSellMaxRow + 1];
    for (int l = 0; l <= kSellMaxRow; ++l) cnt[l] = 0;
    for (int64_t r = r0; r < r1; ++r) cnt[rp[r + 1] - rp[r]]++;
    int at[kSellMaxRow + 1];  // first position of each length, longest first
    int acc = 0;
    for (int l = kSellMaxRow; l >= 0; --l) {
      at[l] = acc;
      acc += cnt[l];
    }
    for (int64_t r = r0; r < r1; ++r) rows[r0 + at[rp[r + 1] - rp[r]]++] = (int32_t)r;
    for (int64_t p = max(r1, r0); p < min(r0 + kSellSigma, npos); ++p) rows[p] = (int32_t)n;
  }
}

// One thread per SELL position (32 * nslices): the column indices (and
// values, when val is given) of the row there, zeros in padding.
__global__ void sell_fill_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                                 int64_t nslices, const int32_t* __restrict__ sptr, int32_t* ci_out,
                                 const void* val, int dt_in, void* val_out, int dt_out,
                                 const int32_t* __restrict__ rmap) {
  const int64_t npos = nslices * 32;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = p >> 5;
    const int lane = (int)(p & 31);
    const int64_t row = sell_row(rmap, p);
    const int64_t off = sptr[sl];
    const int w = (sptr[sl + 1] - sptr[sl]) >> 5;
    const int64_t e0 = row < n ? rp[row] : 0;
    const int len = row < n ? (int)(rp[row + 1] - e0) : 0;
    for (int k = 0; k < w; ++k) {
      const int64_t pos = off + 32 * (int64_t)k + lane;
      if (ci_out) ci_out[pos] = k < len ? ci[e0 + k] : 0;
      if (val_out) st_dt(val_out, dt_out, pos, k < len ? ld_dt(val, dt_in, e0 + k) : 0.0);
    }
  }
}
}  // namespace

int build_sell(const int32_t* rp, const int32_t* ci, int64_t n, int64_t nnz, int32_t max_row, SellData& out,
               cudaStream_t s) {
  out.nslices = 0;
  out.total = 0;
  out.rows.release();
  if (n <= 0 || max_row < 1 || max_row > kSellMaxRow) return SPAI_OK;
  const int64_t ns = (n + 31) / 32;
  if ((int64_t)32 * max_row * ns >= (int64_t)INT32_MAX - 1024) return SPAI_OK;
  int rc;
  DevMem w;
  if ((rc = w.alloc((ns + 1) * sizeof(int32_t), s))) return rc;
  DevMem& sptr = out.sptr;
  if ((rc = sptr.alloc((ns + 1 + 16) * sizeof(int32_t), s))) return rc;
  int32_t total = 0;
  // rows in their own order first; if that pads more than a quarter, rows
  // ordered by length within windows (SELL-C-sigma)
  for (int sorted = 0; sorted < 2; ++sorted) {
    if (sorted) {
      if ((rc = out.rows.alloc((size_t)ns * 32 * sizeof(int32_t), s))) return rc;
      const int64_t nwin = (ns * 32 + kSellSigma - 1) / kSellSigma;
      sell_sort_kernel<<<grid_for(nwin, 128), 128, 0, s>>>(rp, n, ns * 32, out.rows.as<int32_t>()); count_launch();
      SPAI_CUDA(cudaGetLastError());
    }
    SPAI_CUDA(cudaMemsetAsync(w.as<int32_t>() + ns, 0, sizeof(int32_t), s));
    sell_width_kernel<<<grid_for(ns * 32, 256), 256, 0, s>>>(rp, n, ns, w.as<int32_t>(), out.row_map()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    SPAI_CUDA(cudaMemsetAsync(sptr.p, 0, (ns + 1 + 16) * sizeof(int32_t), s));
    if ((rc = exclusive_scan_i32(w.as<int32_t>(), sptr.as<int32_t>(), ns + 1, s))) return rc;
    SPAI_CUDA(cudaMemcpyAsync(&total, sptr.as<int32_t>() + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    if ((int64_t)total * 4 <= nnz * 5) break;  // padding adds at most a quarter
    if (sorted) {
      sptr.release();
      out.rows.release();
      return SPAI_OK;
    }
  }
  const int64_t pad = 64;
  if ((rc = out.ci.alloc((total + pad) * sizeof(int32_t), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(out.ci.p, 0, (total + pad) * sizeof(int32_t), s));
  sell_fill_kernel<<<grid_for(ns * 32, 256), 256, 0, s>>>(rp, ci, n, ns, sptr.as<int32_t>(), out.ci.as<int32_t>(),
                                                          nullptr, 0, nullptr, 0, out.row_map()); count_launch();
  SPAI_CUDA(cudaGetLastError());
  out.sptr.keep();
  out.ci.keep();
  if (out.rows.p) out.rows.keep();
  out.nslices = (int32_t)ns;
  out.total = total;
  out.max_width = max_row;
  return SPAI_OK;
}

int sell_values(const SellData& L, const int32_t* rp, int64_t n, const void* val, int dt_in, void* out, int dt_out,
                cudaStream_t s) {
  if (L.nslices <= 0) return set_error(SPAI_ERR_INVALID, "no SELL layout");
  sell_fill_kernel<<<grid_for((int64_t)L.nslices * 32, 256), 256, 0, s>>>(
      rp, nullptr, n, L.nslices, L.sptr.as<int32_t>(), nullptr, val, dt_in, out, dt_out, L.row_map()); count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

int precond_sell(PrecondData& M, cudaStream_t s) {
  const PatternData& P = *M.P;
  if (P.kind != SPAI_PATTERN_FULL) return SPAI_OK;
  const size_t gs = dtype_size(M.gtype);
  int rc;
  if (P.bsell.nslices > 0) {
    const size_t bb = (size_t)(9 * P.bsell.total + 64) * gs;
    if ((rc = M.bsell_g.alloc(bb, s))) return rc;
    if ((rc = M.bsell_gt.alloc(bb, s))) return rc;
    SPAI_CUDA(cudaMemsetAsync(M.bsell_g.p, 0, bb, s));
    SPAI_CUDA(cudaMemsetAsync(M.bsell_gt.p, 0, bb, s));
    if ((rc = bsell_values(P.bsell, P.g_rp(), P.n, M.g_val.p, M.gtype, M.bsell_g.p, M.gtype, s))) return rc;
    if ((rc = bsell_values(P.bsell, P.gt_rp(), P.n, M.gt_val.p, M.gtype, M.bsell_gt.p, M.gtype, s))) return rc;
    M.bsell_g.keep();
    M.bsell_gt.keep();
  }
  if (P.sell.nslices <= 0) return SPAI_OK;
  const size_t bytes = (size_t)(P.sell.total + 64) * gs;
  if ((rc = M.sell_g.alloc(bytes, s))) return rc;
  if ((rc = M.sell_gt.alloc(bytes, s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(M.sell_g.p, 0, bytes, s));
  SPAI_CUDA(cudaMemsetAsync(M.sell_gt.p, 0, bytes, s));
  if ((rc = sell_values(P.sell, P.g_rp(), P.n, M.g_val.p, M.gtype, M.sell_g.p, M.gtype, s))) return rc;
  if ((rc = sell_values(P.sell, P.gt_rp(), P.n, M.gt_val.p, M.gtype, M.sell_gt.p, M.gtype, s))) return rc;
  M.sell_g.keep();
  M.sell_gt.keep();
  return SPAI_OK;
}

}  // namespace spai

using namespace spai;

extern "C" int spai_build_pattern(const spai_csr* A, int32_t kind, spai_pattern** out, void* stream) {
  if (!out) return set_error(SPAI_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (kind != SPAI_PATTERN_FULL && kind != SPAI_PATTERN_LOWER && kind != SPAI_PATTERN_UPPER)
    return set_error(SPAI_ERR_INVALID, "unknown pattern kind %d", (int)kind);
  if (!A || A->n <= 0) return set_error(SPAI_ERR_INVALID, "A must have n > 0");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  int32_t max_row = 0;
  if ((rc = validate_csr_device(A, true, &max_row, s))) return rc;

  auto P = std::make_shared<PatternData>();
  P->n = A->n;
  P->kind = kind;
  P->a_nnz = A->nnz;
  const int64_t n = A->n;
  const int block = 256;
  DevMem flags;
  if ((rc = flags.alloc(sizeof(int), s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int), s));

  if (kind == SPAI_PATTERN_FULL) {
    P->nnz = A->nnz;
    P->max_row = P->max_row_t = max_row;
    if ((rc = P->rowptr.alloc((n + 1 + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = P->colidx.alloc((A->nnz + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = P->perm.alloc((A->nnz + 1) * sizeof(int32_t), s))) return rc;
    SPAI_CUDA(cudaMemcpyAsync(P->rowptr.p, A->rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    SPAI_CUDA(cudaMemcpyAsync(P->colidx.p, A->colidx, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    perm_kernel<<<grid_for(n, block), block, 0, s>>>(P->g_rp(), P->g_ci(), P->g_rp(), P->g_ci(), n,
                                                     P->perm.as<int32_t>(), flags.as<int>()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    if ((rc = build_sell(P->g_rp(), P->g_ci(), n, A->nnz, max_row, P->sell, s))) return rc;
    if ((rc = build_bsell(P->g_rp(), P->g_ci(), n, A->nnz, P->bsell, s))) return rc;
  } else {
    const int lower_g = (kind == SPAI_PATTERN_LOWER) ? 1 : 0;
    DevMem cnt;
    if ((rc = cnt.alloc((n + 1) * sizeof(int32_t), s))) return rc;
    // G
    if ((rc = P->rowptr.alloc((n + 1 + 16) * sizeof(int32_t), s))) return rc;
    count_tri_kernel<<<grid_for(n, block), block, 0, s>>>(A->rowptr, A->colidx, n, lower_g, cnt.as<int32_t>()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    if ((rc = exclusive_scan_i32(cnt.as<int32_t>(), P->rowptr.as<int32_t>(), n + 1, s))) return rc;
    // G^T: the other triangle (the pattern of A is symmetric)
    if ((rc = P->t_rowptr.alloc((n + 1 + 16) * sizeof(int32_t), s))) return rc;
    count_tri_kernel<<<grid_for(n, block), block, 0, s>>>(A->rowptr, A->colidx, n, 1 - lower_g, cnt.as<int32_t>()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    if ((rc = exclusive_scan_i32(cnt.as<int32_t>(), P->t_rowptr.as<int32_t>(), n + 1, s))) return rc;
    int32_t nnz_g = 0;
    SPAI_CUDA(cudaMemcpyAsync(&nnz_g, P->rowptr.as<int32_t>() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
    P->nnz = nnz_g;
    if ((rc = P->colidx.alloc((nnz_g + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = P->t_colidx.alloc((nnz_g + 16) * sizeof(int32_t), s))) return rc;
    if ((rc = P->src.alloc((nnz_g + 1) * sizeof(int32_t), s))) return rc;
    if ((rc = P->perm.alloc((nnz_g + 1) * sizeof(int32_t), s))) return rc;
    compact_tri_kernel<<<grid_for(n, block), block, 0, s>>>(A->rowptr, A->colidx, n, lower_g, P->rowptr.as<int32_t>(),
                                                            P->colidx.as<int32_t>(), P->src.as<int32_t>()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    compact_tri_kernel<<<grid_for(n, block), block, 0, s>>>(A->rowptr, A->colidx, n, 1 - lower_g,
                                                            P->t_rowptr.as<int32_t>(), P->t_colidx.as<int32_t>(),
                                                            nullptr); count_launch();
    SPAI_CUDA(cudaGetLastError());
    perm_kernel<<<grid_for(n, block), block, 0, s>>>(P->g_rp(), P->g_ci(), P->gt_rp(), P->gt_ci(), n,
                                                     P->perm.as<int32_t>(), flags.as<int>()); count_launch();
    SPAI_CUDA(cudaGetLastError());
    // row lengths bound: a triangle row is no longer than the full row
    P->max_row = P->max_row_t = max_row;
  }
  int hf = 0;
  SPAI_CUDA(cudaMemcpyAsync(&hf, flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  if (hf) return set_error(SPAI_ERR_BAD_CSR, "pattern: %s", flag_text(hf).c_str());
  for (DevMem* m : {&P->rowptr, &P->colidx, &P->t_rowptr, &P->t_colidx, &P->perm, &P->src}) m->keep();
  *out = new spai_pattern{P};
  return SPAI_OK;
}

extern "C" int spai_pattern_info(const spai_pattern* P, int64_t* n, int64_t* nnz_g) {
  if (!P) return set_error(SPAI_ERR_INVALID, "pattern is NULL");
  if (n) *n = P->d->n;
  if (nnz_g) *nnz_g = P->d->nnz;
  return SPAI_OK;
}

extern "C" int spai_pattern_export(const spai_pattern* Ph, int32_t* rowptr, int32_t* colidx, int32_t* t_rowptr,
                                   int32_t* t_colidx, int32_t* perm, void* stream) {
  if (!Ph) return set_error(SPAI_ERR_INVALID, "pattern is NULL");
  const PatternData& P = *Ph->d;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rb = (P.n + 1) * sizeof(int32_t), eb = P.nnz * sizeof(int32_t);
  if (rowptr) SPAI_CUDA(cudaMemcpyAsync(rowptr, P.g_rp(), rb, cudaMemcpyDeviceToDevice, s));
  if (colidx && eb) SPAI_CUDA(cudaMemcpyAsync(colidx, P.g_ci(), eb, cudaMemcpyDeviceToDevice, s));
  if (t_rowptr) SPAI_CUDA(cudaMemcpyAsync(t_rowptr, P.gt_rp(), rb, cudaMemcpyDeviceToDevice, s));
  if (t_colidx && eb) SPAI_CUDA(cudaMemcpyAsync(t_colidx, P.gt_ci(), eb, cudaMemcpyDeviceToDevice, s));
  if (perm && eb) SPAI_CUDA(cudaMemcpyAsync(perm, P.perm.p, eb, cudaMemcpyDeviceToDevice, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  return SPAI_OK;
}

extern "C" void spai_pattern_destroy(spai_pattern* P) { delete P; }
