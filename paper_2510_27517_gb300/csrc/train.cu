// Optimiser step for training the GNN (Sec. 4.1: AdamW with an exponentially
// decaying learning rate, the GNN trained on the SAI loss of Sec. 3.3).
// Decoupled weight decay as Loshchilov & Hutter define it:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   theta -= lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps) + wd theta),
// on a float64 master copy of the weights, written back as the float32 blob
// the forward pass reads.  Optional clipping of g to a 2-norm bound first;
// the norm is one block's fixed-order sum (deterministic).
#include <cmath>

#include "internal.cuh"

namespace spai {
namespace {

constexpr int kNormThreads = 1024;

__global__ void grad_norm_kernel(const double* __restrict__ g, int64_t count, double* out) {
  __shared__ double red[kNormThreads / 32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc = fma(g[i], g[i], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[0] = sqrt(acc);
}

__global__ void adamw_kernel(double* __restrict__ master, double* __restrict__ m, double* __restrict__ v,
                             const double* __restrict__ g, float* __restrict__ blob, int64_t count,
                             spai_adamw_cfg c, double bc1, double bc2, const double* __restrict__ norm) {
  double scale = 1.0;
  if (c.max_grad_norm > 0.0 && norm[0] > c.max_grad_norm) scale = c.max_grad_norm / norm[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double gi = g[i] * scale;
    const double mi = c.beta1 * m[i] + (1.0 - c.beta1) * gi;
    const double vi = c.beta2 * v[i] + (1.0 - c.beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const double mhat = mi / bc1, vhat = vi / bc2;
    const double th = master[i];
    const double nt = th - c.lr * (mhat / (sqrt(vhat) + c.eps) + c.weight_decay * th);
    master[i] = nt;
    blob[i] = (float)nt;
  }
}

}  // namespace
}  // namespace spai

using namespace spai;

extern "C" int spai_adamw_step(double* master, double* m, double* v, const double* grad, float* blob, int64_t count,
                               const spai_adamw_cfg* cfg, int64_t step, double* grad_norm, void* stream) {
  if (!master || !m || !v || !grad || !blob || !cfg) return set_error(SPAI_ERR_INVALID, "null argument");
  if (count < 1 || step < 1) return set_error(SPAI_ERR_INVALID, "count and step must be >= 1");
  if (!(cfg->lr >= 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) ||
      !(cfg->eps > 0.0) || !(cfg->weight_decay >= 0.0))
    return set_error(SPAI_ERR_INVALID, "AdamW needs lr >= 0, 0 <= beta1, beta2 < 1, eps > 0, weight_decay >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  DevMem nrm;
  int rc;
  if ((rc = nrm.alloc(sizeof(double), s))) return rc;
  grad_norm_kernel<<<1, kNormThreads, 0, s>>>(grad, count, nrm.as<double>());
  count_launch();
  const double bc1 = 1.0 - std::pow(cfg->beta1, (double)step);
  const double bc2 = 1.0 - std::pow(cfg->beta2, (double)step);
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  adamw_kernel<<<(unsigned)blocks, 256, 0, s>>>(master, m, v, grad, blob, count, *cfg, bc1, bc2, nrm.as<double>());
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  if (grad_norm) {
    SPAI_CUDA(cudaMemcpyAsync(grad_norm, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPAI_CUDA(cudaStreamSynchronize(s));
  }
  return SPAI_OK;
}
