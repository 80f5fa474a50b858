// SAI loss of a preconditioner (Sec. 3.3, Eqs. 7-8): for k probe vectors w_j
//   L_j = || A (G G^T + eps I) w_j / ||A|| - w_j ||_2^2,
// the Hutchinson estimate of ||A M^-1 / ||A|| - I||_F^2 the paper trains G
// with.  float64 throughout; G in its storage type.  The k probes travel
// together (n x k, probe index fastest), so every stored entry is read once
// for all of them: one warp per row, lane = probe.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace spai {
namespace {

constexpr int kMaxProbes = 32;

// y = M x (+ eps * add) for k right-hand sides; row sums in stored order.
template <class MV>
__global__ void spmm_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const MV* __restrict__ val,
                            const double* __restrict__ x, double* __restrict__ y, int64_t n, int k,
                            const double* __restrict__ add, double eps) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
    if (lane >= k) continue;
    double acc = 0.0;
    for (int e = rp[row]; e < rp[row + 1]; ++e) acc = fma(to_f64(val[e]), x[(int64_t)ci[e] * k + lane], acc);
    if (add) acc = fma(eps, add[row * k + lane], acc);
    y[row * k + lane] = acc;
  }
}

// u = A v, then per probe sum over the block's rows of (u / ||A|| - w)^2:
// block b owns rows [b R, (b + 1) R), warp w its rows w, w + 8, ..., the
// warps' sums are combined in warp order -- a fixed order for any launch.
__global__ void loss_partial_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const double* __restrict__ val, const double* __restrict__ v,
                                    const double* __restrict__ w, const double* __restrict__ anorm, int64_t n, int k,
                                    int64_t rows_per_block, double* part) {
  __shared__ double red[8][kMaxProbes];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double inv = 1.0 / anorm[0];
  const int64_t r0 = blockIdx.x * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  double acc2 = 0.0;
  for (int64_t row = r0 + warp; row < r1; row += 8) {
    if (lane >= k) continue;
    double u = 0.0;
    for (int e = rp[row]; e < rp[row + 1]; ++e) u = fma(val[e], v[(int64_t)ci[e] * k + lane], u);
    const double d = fma(u, inv, -w[row * k + lane]);
    acc2 = fma(d, d, acc2);
  }
  red[warp][lane] = acc2;
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i][threadIdx.x];
    part[blockIdx.x * (int64_t)k + threadIdx.x] = s;
  }
}

__global__ void loss_final_kernel(const double* __restrict__ part, int nb, int k, double* loss) {
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * (int64_t)k + threadIdx.x];
    loss[threadIdx.x] = s;
  }
}

// u = A v / ||A|| - w for k probes (the same arithmetic as the loss).
__global__ void resid_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ val, const double* __restrict__ v,
                             const double* __restrict__ w, const double* __restrict__ anorm, int64_t n, int k,
                             double* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const double inv = 1.0 / anorm[0];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
    if (lane >= k) continue;
    double acc = 0.0;
    for (int e = rp[row]; e < rp[row + 1]; ++e) acc = fma(val[e], v[(int64_t)ci[e] * k + lane], acc);
    u[row * k + lane] = fma(acc, inv, -w[row * k + lane]);
  }
}

// Gradient of the mean loss over the k probes with respect to every stored
// G_ij (G's CSR order): (2 / k) sum_p (a_i y_j + w_i c_j) with a = A u / ||A||
// and c = G^T a passed unscaled (as A u and G^T A u), y = G^T w.  One thread
// per row, probes summed in order.
__global__ void grad_g_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n, int k,
                              const double* __restrict__ au, const double* __restrict__ y,
                              const double* __restrict__ w, const double* __restrict__ cu,
                              const double* __restrict__ anorm, double* __restrict__ grad) {
  const double inv = 1.0 / anorm[0];
  const double scale = 2.0 / (double)k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t j = ci[e];
      double acc = 0.0;
      for (int p = 0; p < k; ++p) {
        const double a = au[i * k + p] * inv, c = cu[j * k + p] * inv;
        acc += a * y[j * k + p] + w[i * k + p] * c;
      }
      grad[e] = scale * acc;
    }
  }
}

template <class MV>
int apply_minv(const PrecondData& M, const double* w, double* t, double* v, int64_t n, int k, cudaStream_t s) {
  const PatternData& P = *M.P;
  const int grid = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  spmm_kernel<MV><<<grid, 256, 0, s>>>(P.gt_rp(), P.gt_ci(), M.gt_val.as<MV>(), w, t, n, k, nullptr, 0.0);
  count_launch();
  spmm_kernel<MV><<<grid, 256, 0, s>>>(P.g_rp(), P.g_ci(), M.g_val.as<MV>(), t, v, n, k, w, M.eps);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

}  // namespace
}  // namespace spai

using namespace spai;

extern "C" int spai_sai_loss(const spai_csr* A, const spai_precond* M, const double* w, int32_t k, double* loss,
                             void* stream) {
  if (!A || !M || !w || !loss) return set_error(SPAI_ERR_INVALID, "null argument");
  if (k < 1 || k > kMaxProbes) return set_error(SPAI_ERR_INVALID, "k must be in 1..%d probes per call", kMaxProbes);
  if (A->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A values must be SPAI_F64");
  const PrecondData& Md = *M->d;
  const int64_t n = A->n;
  if (n <= 0 || Md.P->n != n) return set_error(SPAI_ERR_SHAPE, "A and G sizes differ");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  DevMem tv, nrm, part;
  if ((rc = tv.alloc(2 * (size_t)n * k * sizeof(double), s))) return rc;
  if ((rc = nrm.alloc(sizeof(double), s))) return rc;
  double* t = tv.as<double>();
  double* v = t + n * k;
  if ((rc = matrix_abs_mean(static_cast<const double*>(A->val), A->nnz, nrm.as<double>(), s))) return rc;
  switch (Md.gtype) {
    case SPAI_F64: rc = apply_minv<double>(Md, w, t, v, n, k, s); break;
    case SPAI_F32: rc = apply_minv<float>(Md, w, t, v, n, k, s); break;
    case SPAI_BF16: rc = apply_minv<__nv_bfloat16>(Md, w, t, v, n, k, s); break;
    case SPAI_F16: rc = apply_minv<__half>(Md, w, t, v, n, k, s); break;
    default: return set_error(SPAI_ERR_INVALID, "unknown G storage type");
  }
  if (rc) return rc;
  const int nb = (int)std::min<int64_t>(4 * (int64_t)num_sms(), (n + 7) / 8);
  const int64_t rpb = (n + nb - 1) / nb;
  if ((rc = part.alloc((size_t)nb * k * sizeof(double), s))) return rc;
  loss_partial_kernel<<<nb, 256, 0, s>>>(A->rowptr, A->colidx, static_cast<const double*>(A->val), v, w,
                                          nrm.as<double>(), n, k, rpb, part.as<double>());
  count_launch();
  loss_final_kernel<<<1, 32, 0, s>>>(part.as<double>(), nb, k, loss);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}

extern "C" int spai_sai_loss_grad(const spai_csr* A, const spai_precond* M, const double* w, int32_t k, double* loss,
                                  double* grad_g, void* stream) {
  if (!A || !M || !w || !loss || !grad_g) return set_error(SPAI_ERR_INVALID, "null argument");
  if (k < 1 || k > kMaxProbes) return set_error(SPAI_ERR_INVALID, "k must be in 1..%d probes per call", kMaxProbes);
  if (A->dtype != SPAI_F64) return set_error(SPAI_ERR_INVALID, "A values must be SPAI_F64");
  const PrecondData& Md = *M->d;
  const PatternData& P = *Md.P;
  const int64_t n = A->n;
  if (n <= 0 || P.n != n) return set_error(SPAI_ERR_SHAPE, "A and G sizes differ");
  int rc;
  if ((rc = spai_sai_loss(A, M, w, k, loss, stream))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  DevMem buf, nrm;
  const size_t nk = (size_t)n * k;
  if ((rc = buf.alloc(5 * nk * sizeof(double), s))) return rc;
  if ((rc = nrm.alloc(sizeof(double), s))) return rc;
  double* y = buf.as<double>();  // G^T w
  double* v = y + nk;            // M^-1 w
  double* u = v + nk;            // A v / ||A|| - w
  double* au = u + nk;           // A u (A symmetric: A^T u)
  double* cu = au + nk;          // G^T A u
  if ((rc = matrix_abs_mean(static_cast<const double*>(A->val), A->nnz, nrm.as<double>(), s))) return rc;
  switch (Md.gtype) {
    case SPAI_F64: rc = apply_minv<double>(Md, w, y, v, n, k, s); break;
    case SPAI_F32: rc = apply_minv<float>(Md, w, y, v, n, k, s); break;
    case SPAI_BF16: rc = apply_minv<__nv_bfloat16>(Md, w, y, v, n, k, s); break;
    case SPAI_F16: rc = apply_minv<__half>(Md, w, y, v, n, k, s); break;
    default: return set_error(SPAI_ERR_INVALID, "unknown G storage type");
  }
  if (rc) return rc;
  const int grid = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  const double* av = static_cast<const double*>(A->val);
  resid_kernel<<<grid, 256, 0, s>>>(A->rowptr, A->colidx, av, v, w, nrm.as<double>(), n, k, u);
  count_launch();
  spmm_kernel<double><<<grid, 256, 0, s>>>(A->rowptr, A->colidx, av, u, au, n, k, nullptr, 0.0);
  count_launch();
  switch (Md.gtype) {
    case SPAI_F64:
      spmm_kernel<double><<<grid, 256, 0, s>>>(P.gt_rp(), P.gt_ci(), Md.gt_val.as<double>(), au, cu, n, k, nullptr, 0.0);
      break;
    case SPAI_F32:
      spmm_kernel<float><<<grid, 256, 0, s>>>(P.gt_rp(), P.gt_ci(), Md.gt_val.as<float>(), au, cu, n, k, nullptr, 0.0);
      break;
    case SPAI_BF16:
      spmm_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(P.gt_rp(), P.gt_ci(), Md.gt_val.as<__nv_bfloat16>(), au, cu, n, k,
                                                      nullptr, 0.0);
      break;
    default:
      spmm_kernel<__half><<<grid, 256, 0, s>>>(P.gt_rp(), P.gt_ci(), Md.gt_val.as<__half>(), au, cu, n, k, nullptr, 0.0);
      break;
  }
  count_launch();
  const int gg = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
  grad_g_kernel<<<gg, 256, 0, s>>>(P.g_rp(), P.g_ci(), n, k, au, y, w, cu, nrm.as<double>(), grad_g);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  return SPAI_OK;
}
