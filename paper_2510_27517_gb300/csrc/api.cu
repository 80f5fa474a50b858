// C ABI glue: error state, allocation, handles for preconditioners and
// systems, and the single / batched / host-buffer solve entry points.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include "internal.cuh"

namespace spai {

int engine_tile_nnz(int32_t max_row);
int engine_run(int nsys, SystemData* const* S, PrecondData* const* M, const double* const* b, double* const* x,
               const spai_pcg_opts* o, spai_pcg_result* res, cudaStream_t s, int grid_override, int use_graph);
int engine_tune(SystemData* S, PrecondData* M, bool mixed, cudaStream_t s);

static thread_local std::string g_err = "no error";
static std::atomic<uint64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? SPAI_ERR_OOM : SPAI_ERR_CUDA;
  return set_error(code, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
}

int DevMem::alloc(size_t nbytes, cudaStream_t stream) {
  release();
  if (nbytes == 0) nbytes = 16;
  cudaError_t e = cudaMallocAsync(&p, nbytes, stream);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return cuda_error(e, "cudaMallocAsync");
  }
  bytes = nbytes;
  s = stream;
  return SPAI_OK;
}

void DevMem::release() {
  if (p) {
    if (owned) cudaFree(p);
    else cudaFreeAsync(p, s);
  }
  p = nullptr;
  bytes = 0;
}

size_t dtype_size(int dt) {
  switch (dt) {
    case SPAI_F64: return 8;
    case SPAI_F32: return 4;
    case SPAI_BF16: case SPAI_F16: return 2;
    default: return 0;
  }
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return 1;
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cache[dev] = v;
  }
  return cache[dev];
}

namespace {

__global__ void convert_scatter_kernel(const void* __restrict__ in, int in_t, void* gout, void* gtout, int out_t,
                                       const int32_t* __restrict__ perm, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (in_t == SPAI_F64) ? static_cast<const double*>(in)[i] : (double)static_cast<const float*>(in)[i];
    const int64_t p = perm[i];
    switch (out_t) {
      case SPAI_F64: static_cast<double*>(gout)[i] = v; static_cast<double*>(gtout)[p] = v; break;
      case SPAI_F32: static_cast<float*>(gout)[i] = (float)v; static_cast<float*>(gtout)[p] = (float)v; break;
      case SPAI_BF16: {
        const __nv_bfloat16 h = __double2bfloat16(v);
        static_cast<__nv_bfloat16*>(gout)[i] = h;
        static_cast<__nv_bfloat16*>(gtout)[p] = h;
        break;
      }
      case SPAI_F16: {
        const __half h = __double2half(v);
        static_cast<__half*>(gout)[i] = h;
        static_cast<__half*>(gtout)[p] = h;
        break;
      }
    }
  }
}

__global__ void export_kernel(const void* __restrict__ in, int in_t, void* out, int out_t, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    switch (in_t) {
      case SPAI_F64: v = static_cast<const double*>(in)[i]; break;
      case SPAI_F32: v = static_cast<const float*>(in)[i]; break;
      case SPAI_BF16: v = __bfloat162float(static_cast<const __nv_bfloat16*>(in)[i]); break;
      default: v = __half2float(static_cast<const __half*>(in)[i]); break;
    }
    if (out_t == SPAI_F64) static_cast<double*>(out)[i] = v;
    else static_cast<float*>(out)[i] = (float)v;
  }
}

int grid1(int64_t m) {
  int64_t g = (m + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Tile size heuristic: about `target` nonzeros per tile, with the tile
// count a multiple of the expected co-resident grid so blocks get equal work.
int32_t pick_tile_nnz(int64_t nnz, int64_t grid_est, int64_t target) {
  if (grid_est < 1) grid_est = 1;
  int64_t k = nnz / (grid_est * target);
  if (k < 1) k = 1;
  int64_t t = (nnz + k * grid_est - 1) / (k * grid_est);
  if (t < 256) t = 256;
  if (t > (1 << 20)) t = 1 << 20;
  return (int32_t)t;
}

}  // namespace

int make_precond_from_values(const std::shared_ptr<PatternData>& P, const void* g_val, int val_dtype, int g_dtype,
                             double eps, std::shared_ptr<PrecondData>& out, cudaStream_t s) {
  if (val_dtype != SPAI_F64 && val_dtype != SPAI_F32) return set_error(SPAI_ERR_INVALID, "values must be F64 or F32");
  if (!dtype_size(g_dtype)) return set_error(SPAI_ERR_INVALID, "unknown G dtype");
  if (!(eps >= 0.0)) return set_error(SPAI_ERR_INVALID, "eps must be >= 0");
  auto M = std::make_shared<PrecondData>();
  M->P = P;
  M->gtype = g_dtype;
  M->eps = eps;
  int rc;
  const size_t es = dtype_size(g_dtype);
  if ((rc = M->g_val.alloc((P->nnz + 16) * es, s))) return rc;
  if ((rc = M->gt_val.alloc((P->nnz + 16) * es, s))) return rc;
  M->g_val.keep();
  M->gt_val.keep();
  if (P->nnz > 0) {
    convert_scatter_kernel<<<grid1(P->nnz), 256, 0, s>>>(g_val, val_dtype, M->g_val.p, M->gt_val.p, g_dtype,
                                                         P->perm.as<int32_t>(), P->nnz); count_launch();
    SPAI_CUDA(cudaGetLastError());
  }
  if ((rc = precond_sell(*M, s))) return rc;
  out = M;
  return SPAI_OK;
}

int make_system(const spai_csr* A, int autotune, std::shared_ptr<SystemData>& out, cudaStream_t s);

}  // namespace spai

using namespace spai;

extern "C" const char* spai_last_error(void) { return g_err.c_str(); }

extern "C" const char* spai_version(void) { return "spai-gb300 0.1 (sm_103a)"; }

extern "C" uint64_t spai_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" void spai_pcg_opts_default(spai_pcg_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->max_iter = 0;
  o->replace_period = 50;
  o->criterion = SPAI_CRIT_RESIDUAL;
  o->precision = SPAI_PREC_F64;
  o->inner_rtol = 0.1;
  o->max_outer = 0;
}

extern "C" int spai_precond_from_values(const spai_pattern* P, const void* g_val, int32_t val_dtype, int32_t g_dtype,
                                        double eps, spai_precond** out, void* stream) {
  if (!P || !out || (!g_val && P->d->nnz > 0)) return set_error(SPAI_ERR_INVALID, "null argument");
  *out = nullptr;
  std::shared_ptr<PrecondData> M;
  int rc = make_precond_from_values(P->d, g_val, val_dtype, g_dtype, eps, M, (cudaStream_t)stream);
  if (rc) return rc;
  SPAI_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  *out = new spai_precond{M};
  return SPAI_OK;
}

extern "C" int spai_precond_export(const spai_precond* M, void* g_val, void* gt_val, int32_t dtype, void* stream) {
  if (!M) return set_error(SPAI_ERR_INVALID, "null preconditioner");
  if (dtype != SPAI_F64 && dtype != SPAI_F32) return set_error(SPAI_ERR_INVALID, "export dtype must be F64 or F32");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m = M->d->P->nnz;
  if (m > 0) {
    if (g_val) { export_kernel<<<grid1(m), 256, 0, s>>>(M->d->g_val.p, M->d->gtype, g_val, dtype, m); count_launch(); }
    if (gt_val) { export_kernel<<<grid1(m), 256, 0, s>>>(M->d->gt_val.p, M->d->gtype, gt_val, dtype, m); count_launch(); }
    SPAI_CUDA(cudaGetLastError());
  }
  SPAI_CUDA(cudaStreamSynchronize(s));
  return SPAI_OK;
}

extern "C" int spai_precond_matrix_norm(const spai_precond* M, double* norm) {
  if (!M || !norm) return set_error(SPAI_ERR_INVALID, "null argument");
  *norm = M->d->anorm;
  return SPAI_OK;
}

extern "C" void spai_precond_destroy(spai_precond* M) { delete M; }

namespace spai {
int make_system(const spai_csr* A, int autotune, std::shared_ptr<SystemData>& out, cudaStream_t s) {
  auto S = std::make_shared<SystemData>();
  int rc;
  if ((rc = system_from_csr(A, *S, true, s))) return rc;
  S->rowptr.keep();
  S->colidx.keep();
  S->val64.keep();
  S->val32.keep();
  S->tile_nnz = engine_tile_nnz(S->max_row);
  S->autotune = autotune ? 1 : 0;
  if ((rc = build_sell(S->rowptr.as<int32_t>(), S->colidx.as<int32_t>(), S->n, S->nnz, S->max_row, S->sell_a, s)))
    return rc;
  if (S->sell_a.nslices > 0) {
    const size_t tot = (size_t)S->sell_a.total + 64;
    if ((rc = S->sell_v64.alloc(tot * sizeof(double), s))) return rc;
    if ((rc = S->sell_v32.alloc(tot * sizeof(float), s))) return rc;
    SPAI_CUDA(cudaMemsetAsync(S->sell_v64.p, 0, tot * sizeof(double), s));
    SPAI_CUDA(cudaMemsetAsync(S->sell_v32.p, 0, tot * sizeof(float), s));
    if ((rc = sell_values(S->sell_a, S->rowptr.as<int32_t>(), S->n, S->val64.p, SPAI_F64, S->sell_v64.p, SPAI_F64, s)))
      return rc;
    if ((rc = sell_values(S->sell_a, S->rowptr.as<int32_t>(), S->n, S->val64.p, SPAI_F64, S->sell_v32.p, SPAI_F32, s)))
      return rc;
    S->sell_v64.keep();
    S->sell_v32.keep();
  }
  // rows sorted by length mark an irregular matrix: gathers at random columns,
  // where pairing the vectors read at the same column halves the requests
  S->pair = S->sell_a.rows.p ? 1 : 0;
  if ((rc = build_bsell(S->rowptr.as<int32_t>(), S->colidx.as<int32_t>(), S->n, S->nnz, S->bsell_a, s))) return rc;
  if (S->bsell_a.nslices > 0) {
    const size_t tot = (size_t)9 * S->bsell_a.total + 64;
    if ((rc = S->bsell_v64.alloc(tot * sizeof(double), s))) return rc;
    if ((rc = S->bsell_v32.alloc(tot * sizeof(float), s))) return rc;
    SPAI_CUDA(cudaMemsetAsync(S->bsell_v64.p, 0, tot * sizeof(double), s));
    SPAI_CUDA(cudaMemsetAsync(S->bsell_v32.p, 0, tot * sizeof(float), s));
    if ((rc = bsell_values(S->bsell_a, S->rowptr.as<int32_t>(), S->n, S->val64.p, SPAI_F64, S->bsell_v64.p, SPAI_F64,
                           s)))
      return rc;
    if ((rc = bsell_values(S->bsell_a, S->rowptr.as<int32_t>(), S->n, S->val64.p, SPAI_F64, S->bsell_v32.p, SPAI_F32,
                           s)))
      return rc;
    S->bsell_v64.keep();
    S->bsell_v32.keep();
  }
  out = S;
  return SPAI_OK;
}
}  // namespace spai

extern "C" int spai_system_create(const spai_csr* A, int32_t autotune, spai_system** out, void* stream) {
  if (!out) return set_error(SPAI_ERR_INVALID, "out is NULL");
  *out = nullptr;
  std::shared_ptr<SystemData> S;
  int rc = make_system(A, autotune, S, (cudaStream_t)stream);
  if (rc) return rc;
  SPAI_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  *out = new spai_system{S};
  return SPAI_OK;
}

extern "C" int spai_system_schedule(const spai_system* S, spai_schedule* out) {
  if (!S || !out) return set_error(SPAI_ERR_INVALID, "null argument");
  out->tile_nnz = S->d->tile_nnz;
  out->items_log2 = S->d->items_log2;
  out->staged = S->d->staged;
  out->sell = S->d->sell;
  out->fuse = S->d->fuse;
  out->block = S->d->block;
  out->pair = S->d->pair;
  out->tuned = S->d->tuned;
  return SPAI_OK;
}

extern "C" int spai_system_info(const spai_system* S, spai_system_layout* out) {
  if (!S || !out) return set_error(SPAI_ERR_INVALID, "null argument");
  const SystemData& d = *S->d;
  memset(out, 0, sizeof(*out));
  out->n = d.n;
  out->nnz = d.nnz;
  out->max_row = d.max_row;
  out->sell_slices = d.sell_a.nslices;
  out->sell_total = d.sell_a.total;
  out->sell_sorted = d.sell_a.rows.p ? 1 : 0;
  out->block_slices = d.bsell_a.nslices;
  out->block_total = d.bsell_a.total;
  return SPAI_OK;
}

extern "C" int spai_system_set_schedule(spai_system* S, const spai_schedule* sch) {
  if (!S || !sch) return set_error(SPAI_ERR_INVALID, "null argument");
  SystemData& d = *S->d;
  const int32_t t0 = engine_tile_nnz(d.max_row);
  if (sch->tile_nnz < 0 || sch->tile_nnz > t0)
    return set_error(SPAI_ERR_INVALID, "tile_nnz must be in 1..%d (0: default)", (int)t0);
  if (sch->items_log2 < -4 || sch->items_log2 > 4) return set_error(SPAI_ERR_INVALID, "items_log2 must be in -4..4");
  if ((sch->staged != 0 && sch->staged != 1) || (sch->sell != 0 && sch->sell != 1) ||
      (sch->fuse != 0 && sch->fuse != 1) || (sch->block != 0 && sch->block != 1) ||
      (sch->pair != 0 && sch->pair != 1))
    return set_error(SPAI_ERR_INVALID, "staged, sell, fuse, block and pair must be 0 or 1");
  d.tile_nnz = sch->tile_nnz ? sch->tile_nnz : t0;
  d.items_log2 = sch->items_log2;
  d.staged = sch->staged;
  d.sell = sch->sell;
  d.fuse = sch->fuse;
  d.block = sch->block;
  d.pair = sch->pair;
  d.tuned = 1;
  return SPAI_OK;
}

namespace {
// Tunes (once) every system created with autotune that has not been tuned yet.
int tune_pending(int nsys, SystemData* const* S, PrecondData* const* M, const spai_pcg_opts* o, cudaStream_t s) {
  for (int i = 0; i < nsys; ++i) {
    if (!S[i]->autotune || S[i]->tuned) continue;
    int rc = engine_tune(S[i], M[i], o->precision == SPAI_PREC_MIXED, s);
    if (rc) return rc;
  }
  return SPAI_OK;
}
}  // namespace

extern "C" void spai_system_destroy(spai_system* S) { delete S; }

extern "C" int spai_system_solve(spai_system* S, const spai_precond* M, const double* b, double* x,
                                 const spai_pcg_opts* opts, spai_pcg_result* res, void* stream) {
  if (!S || !M || !b || !x || !opts || !res) return set_error(SPAI_ERR_INVALID, "null argument");
  SystemData* sp = S->d.get();
  PrecondData* mp = M->d.get();
  if (mp->P->n != sp->n) return set_error(SPAI_ERR_SHAPE, "G and A sizes differ");
  int rc = tune_pending(1, &sp, &mp, opts, (cudaStream_t)stream);
  if (rc) return rc;
  return engine_run(1, &sp, &mp, &b, &x, opts, res, (cudaStream_t)stream, 0, 0);
}

extern "C" int spai_pcg_solve(const spai_csr* A, const spai_precond* M, const double* b, double* x,
                              const spai_pcg_opts* opts, spai_pcg_result* res, void* stream) {
  if (!A || !M || !b || !x || !opts || !res) return set_error(SPAI_ERR_INVALID, "null argument");
  std::shared_ptr<SystemData> S;
  int rc = make_system(A, 0, S, (cudaStream_t)stream);
  if (rc) return rc;
  SystemData* sp = S.get();
  PrecondData* mp = M->d.get();
  rc = engine_run(1, &sp, &mp, &b, &x, opts, res, (cudaStream_t)stream, 0, 0);
  cudaStreamSynchronize((cudaStream_t)stream);
  return rc;
}

extern "C" int spai_pcg_solve_batched(int32_t nsys, spai_system* const* S, const spai_precond* const* M,
                                      const double* const* b, double* const* x, const spai_pcg_opts* opts,
                                      spai_pcg_result* res, void* stream) {
  if (nsys <= 0 || !S || !M || !b || !x || !opts || !res) return set_error(SPAI_ERR_INVALID, "null argument");
  std::vector<SystemData*> sp(nsys);
  std::vector<PrecondData*> mp(nsys);
  for (int i = 0; i < nsys; ++i) {
    if (!S[i] || !M[i]) return set_error(SPAI_ERR_INVALID, "null system or preconditioner %d", i);
    sp[i] = S[i]->d.get();
    mp[i] = M[i]->d.get();
  }
  spai_pcg_opts o = *opts;
  o.record_history = 0;
  for (int i = 0; i < nsys; ++i)
    if (mp[i]->P->n != sp[i]->n) return set_error(SPAI_ERR_SHAPE, "G and A sizes differ (system %d)", i);
  int rc = tune_pending(nsys, sp.data(), mp.data(), &o, (cudaStream_t)stream);
  if (rc) return rc;
  return engine_run(nsys, sp.data(), mp.data(), b, x, &o, res, (cudaStream_t)stream, 0, 1);
}

extern "C" int spai_pcg_solve_host(const spai_csr* A, const spai_precond* M, const double* b_host, double* x_host,
                                   const spai_pcg_opts* opts, spai_pcg_result* res, void* stream) {
  if (!A || !M || !b_host || !x_host || !opts || !res) return set_error(SPAI_ERR_INVALID, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n;
  DevMem db, dx;
  int rc;
  if ((rc = db.alloc(n * sizeof(double), s))) return rc;
  if ((rc = dx.alloc(n * sizeof(double), s))) return rc;
  SPAI_CUDA(cudaMemcpyAsync(db.p, b_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  SPAI_CUDA(cudaMemcpyAsync(dx.p, x_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  rc = spai_pcg_solve(A, M, db.as<double>(), dx.as<double>(), opts, res, stream);
  if (rc != SPAI_OK && rc != SPAI_ERR_NOT_CONVERGED && rc != SPAI_ERR_BREAKDOWN) return rc;
  SPAI_CUDA(cudaMemcpyAsync(x_host, dx.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  SPAI_CUDA(cudaStreamSynchronize(s));
  return rc;
}
