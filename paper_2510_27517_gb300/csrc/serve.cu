// Continuous-batching solve server.
//
// Requests (b, x in host memory) are queued by spai_server_submit.  A worker
// thread owns a CUDA stream and loops:
//   admit   queued requests into free slots while the device bytes of the
//           admitted requests stay under hbm_cap_bytes (copy b to the device);
//   run     one persistent launch of the PCG engine over every live request
//           for at most chunk_iters iterations (systems of any size share the
//           launch; each keeps its own scalars and state machine);
//   retire  requests whose state reached DONE: copy x to the host, compute
//           the float64 true residual, record the completion.
// A request stops taking device work in the phase it converges; new requests
// join at the next launch.  Each system's reductions depend only on that
// system, so a request's result is the same alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "internal.cuh"

namespace spai {

int engine_true_residuals(int nsys, SystemData* const* S, const double* const* b, double* const* x, double* out,
                          cudaStream_t s);

namespace {

struct Request {
  uint64_t ticket = 0;
  int64_t sys = 0;
  const double* bh = nullptr;
  double* xh = nullptr;
  double t_submit = 0, t_admit = 0;
  size_t bytes = 0;
  int32_t pair = 0;  // vector layout of the workspace (the system's schedule at submission)
  DevMem buf;  // b, x, engine workspace
  std::vector<unsigned char> state;
};

}  // namespace

struct ServerImpl {
  spai_serve_cfg cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::pair<std::shared_ptr<SystemData>, std::shared_ptr<PrecondData>>> systems;
  std::deque<std::unique_ptr<Request>> queue;
  std::deque<spai_completion> done;
  std::map<uint64_t, spai_completion> done_by_ticket;
  uint64_t next_ticket = 1;
  bool stop = false;
  int worker_error = 0;
  std::string worker_msg;
  std::thread worker;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now_us() const {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  int loop(cudaStream_t s);
};

int ServerImpl::loop(cudaStream_t s) {
  const bool mixed = cfg.opts.precision == SPAI_PREC_MIXED;
  EngineSession* es = nullptr;
  std::vector<std::unique_ptr<Request>> live;
  size_t live_bytes = 0;
  int rc = SPAI_OK;
  bool dirty = false;
  const int chunk_iters = cfg.chunk_iters > 0 ? cfg.chunk_iters : 16;
  const int max_slots = cfg.max_slots > 0 ? cfg.max_slots : 64;
  auto member = [&](Request& r) {
    SessionMember m;
    m.S = systems[r.sys].first.get();
    m.M = systems[r.sys].second.get();
    const size_t nb = m.S->n * sizeof(double);
    m.b = r.buf.as<double>();
    m.x = reinterpret_cast<double*>(r.buf.as<char>() + nb);
    m.work = r.buf.as<char>() + 2 * nb;
    m.pair = r.pair;
    m.state = r.state;
    return m;
  };
  for (;;) {
    // ---- admission, in arrival order, by device footprint ----
    {
      std::unique_lock<std::mutex> lk(mu);
      if (live.empty() && queue.empty()) {
        if (stop) break;
        cv_work.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      while (!queue.empty() && (int)live.size() < max_slots) {
        if (live_bytes + queue.front()->bytes > (size_t)cfg.hbm_cap_bytes && !live.empty()) break;
        std::unique_ptr<Request> r = std::move(queue.front());
        queue.pop_front();
        SystemData& S = *systems[r->sys].first;
        const size_t nb = S.n * sizeof(double);
        if ((rc = r->buf.alloc(2 * nb + engine_work_bytes(S.n, mixed, r->pair != 0), s))) break;
        double* bd = r->buf.as<double>();
        if (cudaMemcpyAsync(bd, r->bh, nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(reinterpret_cast<char*>(bd) + nb, 0, nb, s) != cudaSuccess) {
          rc = set_error(SPAI_ERR_CUDA, "server: copy of b failed");
          break;
        }
        r->t_admit = now_us();
        live_bytes += r->bytes;
        live.push_back(std::move(r));
        dirty = true;
      }
      if (rc) break;
    }
    if (live.empty()) continue;
    // ---- one persistent launch over every live request ----
    if (!es && (rc = session_create(mixed, systems[live[0]->sys].second->gtype, cfg.opts, s, &es))) break;
    std::vector<SessionMember> mem;
    mem.reserve(live.size());
    for (auto& r : live) mem.push_back(member(*r));
    if (dirty) {
      if ((rc = session_set(es, mem))) break;
      dirty = false;
    }
    if ((rc = session_launch(es, 3 * chunk_iters + 4))) break;
    std::vector<SessionView> views;
    if ((rc = session_read(es, mem, views))) break;
    std::vector<size_t> fin;
    for (size_t i = 0; i < live.size(); ++i) {
      live[i]->state = mem[i].state;
      if (views[i].done) fin.push_back(i);
    }
    if (fin.empty()) continue;
    // ---- retire converged requests ----
    std::vector<SystemData*> Ss;
    std::vector<const double*> bs;
    std::vector<double*> xs;
    for (size_t k : fin) {
      Ss.push_back(mem[k].S);
      bs.push_back(mem[k].b);
      xs.push_back(mem[k].x);
    }
    std::vector<double> tr(fin.size());
    if ((rc = engine_true_residuals((int)fin.size(), Ss.data(), bs.data(), xs.data(), tr.data(), s))) break;
    for (size_t j = 0; j < fin.size(); ++j) {
      if (cudaMemcpyAsync(live[fin[j]]->xh, xs[j], Ss[j]->n * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess) {
        rc = set_error(SPAI_ERR_CUDA, "server: copy of x failed");
        break;
      }
    }
    if (rc) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(SPAI_ERR_CUDA, "server: copy of x failed"); break; }
    std::vector<std::unique_ptr<Request>> keep;
    std::vector<spai_completion> comps;
    for (size_t i = 0, j = 0; i < live.size(); ++i) {
      if (j < fin.size() && fin[j] == i) {
        spai_completion c;
        memset(&c, 0, sizeof(c));
        c.ticket = live[i]->ticket;
        c.status = views[i].status;
        c.iters = views[i].iters;
        c.outer_iters = views[i].outer;
        c.true_rel_res = tr[j];
        c.t_submit_us = live[i]->t_submit;
        c.t_admit_us = live[i]->t_admit;
        c.t_done_us = now_us();
        comps.push_back(c);
        live_bytes -= live[i]->bytes;
        ++j;
      } else {
        keep.push_back(std::move(live[i]));
      }
    }
    live.swap(keep);
    keep.clear();  // frees the retired requests' device buffers (stream-ordered)
    dirty = true;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& c : comps) {
        done.push_back(c);
        done_by_ticket[c.ticket] = c;
      }
    }
    cv_done.notify_all();
  }
  if (es) session_destroy(es);
  return rc;
}

void ServerImpl::run() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    worker_error = SPAI_ERR_CUDA;
    worker_msg = "server: cannot create a stream";
    cv_done.notify_all();
    return;
  }
  int rc = loop(s);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (rc != SPAI_OK) {
    std::lock_guard<std::mutex> lk(mu);
    worker_error = rc;
    worker_msg = spai_last_error();
  }
  cv_done.notify_all();
}

}  // namespace spai

struct spai_server {
  spai::ServerImpl impl;
};

using namespace spai;

extern "C" int spai_server_create(const spai_serve_cfg* cfg, spai_server** out) {
  if (!cfg || !out) return set_error(SPAI_ERR_INVALID, "null argument");
  *out = nullptr;
  if (cfg->hbm_cap_bytes <= 0) return set_error(SPAI_ERR_INVALID, "hbm_cap_bytes must be positive");
  if (cfg->opts.precision != SPAI_PREC_F64 && cfg->opts.precision != SPAI_PREC_MIXED)
    return set_error(SPAI_ERR_INVALID, "unknown precision");
  auto* srv = new spai_server();
  srv->impl.cfg = *cfg;
  srv->impl.cfg.opts.record_history = 0;
  srv->impl.cfg.opts.history = nullptr;
  cudaGetDevice(&srv->impl.device);
  srv->impl.worker = std::thread([srv] { srv->impl.run(); });
  *out = srv;
  return SPAI_OK;
}

extern "C" int spai_server_register(spai_server* srv, spai_system* S, const spai_precond* M, int64_t* sys_id) {
  if (!srv || !S || !M || !sys_id) return set_error(SPAI_ERR_INVALID, "null argument");
  if (M->d->P->n != S->d->n) return set_error(SPAI_ERR_SHAPE, "G and A sizes differ");
  std::lock_guard<std::mutex> lk(srv->impl.mu);
  for (auto& sp : srv->impl.systems)
    if (sp.second->gtype != M->d->gtype) return set_error(SPAI_ERR_INVALID, "all preconditioners need one G type");
  srv->impl.systems.push_back({S->d, M->d});
  *sys_id = (int64_t)srv->impl.systems.size() - 1;
  return SPAI_OK;
}

extern "C" int spai_server_submit(spai_server* srv, int64_t sys_id, const double* b_host, double* x_host,
                                  uint64_t* ticket) {
  if (!srv || !b_host || !x_host || !ticket) return set_error(SPAI_ERR_INVALID, "null argument");
  ServerImpl& I = srv->impl;
  std::unique_ptr<Request> r(new Request());
  {
    std::lock_guard<std::mutex> lk(I.mu);
    if (I.worker_error) return set_error(I.worker_error, "server worker failed: %s", I.worker_msg.c_str());
    if (sys_id < 0 || sys_id >= (int64_t)I.systems.size()) return set_error(SPAI_ERR_NOT_FOUND, "unknown system id");
    const int64_t n = I.systems[sys_id].first->n;
    const bool mixed = I.cfg.opts.precision == SPAI_PREC_MIXED;
    r->pair = I.systems[sys_id].first->pair;
    r->bytes = 2 * n * sizeof(double) + engine_work_bytes(n, mixed, r->pair != 0);
    if ((int64_t)r->bytes > I.cfg.hbm_cap_bytes)
      return set_error(SPAI_ERR_TOO_LARGE, "request needs %zu device bytes, cap is %lld", r->bytes,
                       (long long)I.cfg.hbm_cap_bytes);
    r->ticket = I.next_ticket++;
    r->sys = sys_id;
    r->bh = b_host;
    r->xh = x_host;
    r->t_submit = I.now_us();
    *ticket = r->ticket;
    I.queue.push_back(std::move(r));
  }
  I.cv_work.notify_one();
  return SPAI_OK;
}

extern "C" int spai_server_poll(spai_server* srv, spai_completion* out, int32_t max, int32_t* count) {
  if (!srv || !count || (max > 0 && !out)) return set_error(SPAI_ERR_INVALID, "null argument");
  ServerImpl& I = srv->impl;
  std::lock_guard<std::mutex> lk(I.mu);
  int k = 0;
  while (k < max && !I.done.empty()) {
    out[k++] = I.done.front();
    I.done.pop_front();
  }
  *count = k;
  if (I.worker_error && k == 0) return set_error(I.worker_error, "server worker failed: %s", I.worker_msg.c_str());
  return SPAI_OK;
}

extern "C" int spai_server_wait(spai_server* srv, uint64_t ticket, int64_t timeout_ms, spai_completion* out) {
  if (!srv || !out) return set_error(SPAI_ERR_INVALID, "null argument");
  ServerImpl& I = srv->impl;
  std::unique_lock<std::mutex> lk(I.mu);
  if (ticket == 0 || ticket >= I.next_ticket) return set_error(SPAI_ERR_NOT_FOUND, "unknown ticket");
  const bool ok = I.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] {
    return I.done_by_ticket.count(ticket) > 0 || I.worker_error != 0;
  });
  if (I.done_by_ticket.count(ticket)) {
    *out = I.done_by_ticket[ticket];
    return SPAI_OK;
  }
  if (I.worker_error) return set_error(I.worker_error, "server worker failed: %s", I.worker_msg.c_str());
  (void)ok;
  return set_error(SPAI_ERR_TIMEOUT, "request %llu not finished within %lld ms", (unsigned long long)ticket,
                   (long long)timeout_ms);
}

extern "C" int spai_server_destroy(spai_server* srv) {
  if (!srv) return SPAI_OK;
  {
    std::lock_guard<std::mutex> lk(srv->impl.mu);
    srv->impl.stop = true;
  }
  srv->impl.cv_work.notify_all();
  if (srv->impl.worker.joinable()) srv->impl.worker.join();
  const int err = srv->impl.worker_error;
  delete srv;
  return err ? set_error(err, "server worker had failed") : SPAI_OK;
}
