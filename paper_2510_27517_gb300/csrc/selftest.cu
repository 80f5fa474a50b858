// Self-test of the bounded device-side waits the persistent solver relies on:
// a grid barrier that one block too many is expected at (so nobody releases
// it), an mbarrier that nothing arrives on, and an item-flag wait (the order
// of the two passes of a fused step) on flags nothing publishes.  Each must
// give up after the limit, flag SPAI_ERR_TIMEOUT and let the kernel return,
// leaving the context usable.  The paper has no counterpart; this checks failure detection
// without faulting or hanging the GPU.
#include "internal.cuh"

namespace spai {
namespace {

__global__ void wait_timeout_kernel(GridSync* g, uint64_t limit_ns, int* out, const unsigned* flags, int* ferr) {
  __shared__ int sflag;
  __shared__ uint64_t bar;
  const int ex = grid_barrier(g, gridDim.x + 1, limit_ns, &sflag);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool arrived = mbar_wait_bounded(&bar, 0, limit_ns);
  // 40 flags (two polling rounds of warp 0), all still 0: epoch 1 never comes
  wait_items(ItemWait{flags, 0, 39, 1u}, limit_ns, ferr);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = *(volatile int*)&g->err;
    out[1] = arrived ? 1 : 0;
    out[2] = ex;
  }
}

}  // namespace
}  // namespace spai

using namespace spai;

extern "C" int spai_selftest_wait_timeout(int64_t limit_us, int32_t* detected, void* stream) {
  if (!detected || limit_us <= 0 || limit_us > 1000000)
    return set_error(SPAI_ERR_INVALID, "limit_us must be in 1..1000000 and detected non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DevMem buf;
  int rc;
  // [GridSync | out: 4 ints | flag-wait error: 1 int, padded | 40 flags]
  const size_t bytes = sizeof(GridSync) + 64 + 40 * sizeof(unsigned);
  if ((rc = buf.alloc(bytes, s))) return rc;
  SPAI_CUDA(cudaMemsetAsync(buf.p, 0, bytes, s));
  GridSync* g = buf.as<GridSync>();
  int* out = reinterpret_cast<int*>(buf.as<char>() + sizeof(GridSync));
  int* ferr = out + 4;
  const unsigned* flags = reinterpret_cast<const unsigned*>(buf.as<char>() + sizeof(GridSync) + 64);
  // two blocks, both resident on any GPU: the barrier still never completes
  wait_timeout_kernel<<<2, 64, 0, s>>>(g, (uint64_t)limit_us * 1000ull, out, flags, ferr);
  count_launch();
  SPAI_CUDA(cudaGetLastError());
  int h[5] = {0, 0, 0, 0, 0};
  SPAI_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  *detected = (h[0] == SPAI_ERR_TIMEOUT && h[1] == 0 && h[2] == 1 && h[4] == SPAI_ERR_TIMEOUT) ? 1 : 0;
  return SPAI_OK;
}
