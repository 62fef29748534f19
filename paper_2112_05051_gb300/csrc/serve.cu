// Request server: many backward-Euler time-step solves (Sec. 3's step, one per
// request) in flight on one GPU at once.
//
// Structure.  `slots` host worker threads, each owning one CUDA stream.  A
// worker takes the oldest queued request that can be admitted, runs it with the
// ordinary entry points (rich_create / rich_step / rich_destroy) on its own
// stream and records host timestamps.  Because every device allocation of the
// library is stream-ordered (cudaMallocAsync on the context's stream) and the
// only host waits are on the worker's own stream, the kernels of the requests
// in flight interleave on the device and a request never waits for another one
// to finish.  Each request runs exactly the kernels a lone rich_step would run,
// with the same fixed-order reductions, so its result does not depend on the mix.
//
// Admission.  A request is admitted in arrival order (requests of a busy
// session are passed over until the session is free) when a slot is free and
// its device-memory estimate fits in the budget beside the requests in flight
// and the resident sessions; idle sessions are evicted least recently used
// first to make room.  The estimate (per cell: context arrays, Krylov vectors,
// hierarchy, product lists) is deliberately generous; `mem_in_flight` in each
// result reports what was reserved when it was admitted.
//
// Sessions.  A request with a session id keeps its context (pressure, K_s field,
// AMG hierarchy) on the device after it finishes; the next request of the
// session continues from that pressure (p0_host NULL) and reuses the hierarchy.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace rich {

struct SrvRequest {
  long long id = 0;
  rich_request r{};
  double est = 0.0;
  bool done = false;
  rich_request_result res{};
};

struct SrvSession {
  long long id = 0;
  rich_ctx* ctx = nullptr;
  double* p = nullptr;
  double est = 0.0;
  bool busy = false;
  long long last_use = 0;
  rich_request shape{};  // grid, soil, kmean, bc, precision of the first request
};

}  // namespace rich

struct rich_server {
  int device = 0;
  rich_server_opts o{};
  double budget = 0.0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<rich::SrvRequest*> queue;
  std::unordered_map<long long, rich::SrvRequest*> reqs;
  std::unordered_map<long long, rich::SrvSession*> sessions;
  double reserved = 0.0;  // admitted one-off requests plus resident sessions
  int in_flight = 0, max_in_flight = 0;
  long long admitted = 0, next_id = 1, use_clock = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  // batched members and their failures per class (grid, mean, precision): a class
  // whose members fail often is served alone (a failed member costs its batch
  // attempt and a lone rerun)
  std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> batch_record;
};

namespace rich {

static double srv_now(const rich_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Device bytes a request may hold: context arrays (constitutive values, the two
// 7-point stencils, the finest CSR, Newton vectors), Krylov vectors, the AMG
// hierarchy with its FP32 copies, the Galerkin product lists, plus a fixed margin.
static double srv_estimate(const rich_request& r) {
  double n = (double)r.grid.nx * r.grid.ny * r.grid.nz;
  double vec = r.opts.krylov.kind == RICH_KRYLOV_FGMRES ? 2.0 * r.opts.krylov.restart + 8.0
                                                        : 8.0 + 2.0 * r.opts.fcg_fallback_restart;
  double per = 1000.0 + 8.0 * vec + (r.precision == RICH_PREC_MIXED ? 200.0 : 0.0) +
               (r.opts.amg.product_lists ? 800.0 : 0.0);
  return n * per + 64.0 * 1024 * 1024;
}

static bool srv_same_shape(const rich_request& a, const rich_request& b) {
  if (a.grid.nx != b.grid.nx || a.grid.ny != b.grid.ny || a.grid.nz != b.grid.nz) return false;
  if (a.grid.lx != b.grid.lx || a.grid.ly != b.grid.ly || a.grid.lz != b.grid.lz) return false;
  if (a.grid.h[0] != b.grid.h[0] || a.grid.h[1] != b.grid.h[1] || a.grid.h[2] != b.grid.h[2]) return false;
  if (a.kmean != b.kmean || a.precision != b.precision) return false;
  if (memcmp(a.bc.kind, b.bc.kind, sizeof(a.bc.kind)) || memcmp(a.bc.value, b.bc.value, sizeof(a.bc.value)))
    return false;
  return a.soil.alpha == b.soil.alpha && a.soil.beta == b.soil.beta && a.soil.theta_s == b.soil.theta_s &&
         a.soil.theta_r == b.soil.theta_r && a.soil.a == b.soil.a && a.soil.gamma == b.soil.gamma &&
         a.soil.ks_const == b.soil.ks_const && a.soil.rho_phi == b.soil.rho_phi;
}

// Frees a session's device state on the caller's (idle) stream.
static void srv_free_session(SrvSession* se, cudaStream_t st) {
  if (se->ctx) {
    se->ctx->st = st;
    AllocStream guard(st);
    dfree(se->p);
    rich_destroy(se->ctx);
  }
  delete se;
}

// Under s->mu: the next admissible request, or nullptr.  Evicted sessions are
// appended to *evict (freed by the caller outside the lock).
static SrvRequest* srv_pick(rich_server* s, std::vector<SrvSession*>* evict) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    SrvRequest* q = *it;
    SrvSession* se = nullptr;
    if (q->r.session) {
      auto f = s->sessions.find(q->r.session);
      if (f != s->sessions.end()) {
        se = f->second;
        if (se->busy) continue;  // a later request of another problem may go first
      }
    }
    double need = (q->r.session && se) ? 0.0 : q->est;
    bool new_session = q->r.session && !se;
    auto lru_idle = [&]() -> SrvSession* {
      SrvSession* v = nullptr;
      for (auto& kv : s->sessions)
        if (!kv.second->busy && kv.second != se && (!v || kv.second->last_use < v->last_use)) v = kv.second;
      return v;
    };
    while (s->reserved + need > s->budget ||
           (new_session && s->o.max_sessions > 0 && (int)s->sessions.size() >= s->o.max_sessions)) {
      SrvSession* v = lru_idle();
      if (!v) break;
      s->sessions.erase(v->id);
      s->reserved -= v->est;
      evict->push_back(v);
    }
    if (s->reserved + need > s->budget) return nullptr;  // head of line waits for memory
    if (new_session && s->o.max_sessions > 0 && (int)s->sessions.size() >= s->o.max_sessions) return nullptr;
    s->queue.erase(it);
    s->reserved += need;
    if (new_session) {
      se = new SrvSession();
      se->id = q->r.session;
      se->est = q->est;
      se->shape = q->r;
      s->sessions[se->id] = se;
    }
    if (se) {
      se->busy = true;
      se->last_use = ++s->use_clock;
    }
    return q;
  }
  return nullptr;
}

// Whether request b may be stepped in one batch with request a (rich_step_batch).
constexpr int kBatchRecordMin = 16;        // members recorded before a class can be taken out of batching
constexpr double kBatchFailMax = 0.25;     // failure fraction above which it is

static std::tuple<int, int, int, int, int> srv_class(const rich_request& r) {
  return std::make_tuple(r.grid.nx, r.grid.ny, r.grid.nz, r.kmean, r.precision);
}

static bool srv_batchable(const rich_server* s, const rich_request& a, const rich_request& b) {
  if (a.session || b.session || !a.p0_host || !b.p0_host) return false;
  if ((long long)a.grid.nx * a.grid.ny * a.grid.nz > s->o.batch_min_cells) return false;
  auto rec = s->batch_record.find(srv_class(a));
  if (rec != s->batch_record.end() && rec->second.first >= kBatchRecordMin &&
      rec->second.second > kBatchFailMax * rec->second.first)
    return false;
  if (!srv_same_shape(a, b) || a.dt != b.dt) return false;
  if ((a.ks_field_host == nullptr) != (b.ks_field_host == nullptr)) return false;
  if (a.opts.krylov.kind != RICH_KRYLOV_FCG || a.opts.max_dt_halvings != 0) return false;
  return memcmp(&a.opts, &b.opts, sizeof(a.opts)) == 0;
}

// Under s->mu: queued one-off requests that can join q's batch and fit the budget.
static void srv_pick_mates(rich_server* s, SrvRequest* q, std::vector<SrvRequest*>* mates) {
  if (s->o.batch_max <= 1) return;
  for (auto it = s->queue.begin(); it != s->queue.end() && (int)mates->size() + 1 < s->o.batch_max;) {
    SrvRequest* m = *it;
    if (srv_batchable(s, q->r, m->r) && s->reserved + m->est <= s->budget) {
      s->reserved += m->est;
      mates->push_back(m);
      it = s->queue.erase(it);
    } else {
      ++it;
    }
  }
}

static void srv_run(SrvRequest* q, SrvSession* se, cudaStream_t st);

// Steps q and its mates as one batch; a member whose step fails is rerun alone.
static void srv_run_batch(rich_server* s, std::vector<SrvRequest*>& qs, cudaStream_t st) {
  const rich_request& r0 = qs[0]->r;
  const int B = (int)qs.size();
  const long long n = (long long)r0.grid.nx * r0.grid.ny * r0.grid.nz;
  int status = RICH_OK;
  {
    AllocStream guard(st);
    double* ks = nullptr;
    double* p = nullptr;
    rich_ctx* c = nullptr;
    if (r0.ks_field_host) {
      status = dalloc(&ks, n * B);
      for (int b = 0; b < B && !status; ++b)
        if (cudaMemcpyAsync(ks + b * n, qs[b]->r.ks_field_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
          status = RICH_ECUDA;
    }
    rich_soil so = r0.soil;
    so.ks_field_dev = ks;
    if (!status) status = rich_create_batch(&r0.grid, B, &so, r0.kmean, &r0.bc, r0.precision, st, &c);
    dfree(ks);
    if (!status) status = dalloc(&p, n * B);
    for (int b = 0; b < B && !status; ++b)
      if (cudaMemcpyAsync(p + b * n, qs[b]->r.p0_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        status = RICH_ECUDA;
    std::vector<rich_step_stats> stats(B);
    std::vector<int> stb(B, RICH_ECUDA);
    if (!status) status = rich_step_batch(c, p, r0.dt, &r0.opts, stats.data(), stb.data());
    for (int b = 0; b < B; ++b) {
      qs[b]->res.batch_size = B;
      qs[b]->res.batch_rerun = 0;
      if (status || stb[b] != RICH_OK) continue;
      if (qs[b]->r.p_out_host &&
          cudaMemcpyAsync(qs[b]->r.p_out_host, p + b * n, sizeof(double) * n, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess)
        stb[b] = RICH_ECUDA;
      qs[b]->res.status = stb[b];
      qs[b]->res.stats = stats[b];
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && !status) status = RICH_ECUDA;
    dfree(p);
    if (c) rich_destroy(c);
    int failed = 0;
    for (int b = 0; b < B; ++b)
      if (status || stb[b] != RICH_OK) {
        qs[b]->res.batch_rerun = 1;
        ++failed;
      }
    std::lock_guard<std::mutex> lock(s->mu);
    auto& rec = s->batch_record[srv_class(r0)];
    rec.first += B;
    rec.second += failed;
  }
  for (int b = 0; b < B; ++b)
    if (qs[b]->res.batch_rerun) srv_run(qs[b], nullptr, st);  // the lone path decides its result
}

static void srv_run(SrvRequest* q, SrvSession* se, cudaStream_t st) {
  const rich_request& r = q->r;
  AllocStream guard(st);
  long long n = (long long)r.grid.nx * r.grid.ny * r.grid.nz;
  int status = RICH_OK;
  rich_ctx* c = nullptr;
  double* p = nullptr;
  rich_step_stats stats{};
  const bool resident = se && se->ctx;  // a session state left by an earlier request
  if (resident) {
    if (!srv_same_shape(se->shape, r)) status = RICH_EINVAL;
    c = se->ctx;
    c->st = st;
    p = se->p;
  } else if (!r.p0_host) {
    status = RICH_ESTATE;  // nothing to continue from (the session was evicted or never ran)
  } else {
    double* ks = nullptr;
    if (r.ks_field_host) {
      status = dalloc(&ks, n);
      if (!status && cudaMemcpyAsync(ks, r.ks_field_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) !=
                         cudaSuccess)
        status = RICH_ECUDA;
    }
    rich_soil so = r.soil;
    so.ks_field_dev = ks;
    if (!status) status = rich_create(&r.grid, &so, r.kmean, &r.bc, r.precision, st, &c);
    dfree(ks);
    if (!status) status = dalloc(&p, n);
    if (se && !status) {
      se->ctx = c;
      se->p = p;
    }
  }
  if (!status && r.p0_host &&
      cudaMemcpyAsync(p, r.p0_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    status = RICH_ECUDA;
  bool stepped = false;
  if (!status) {
    status = rich_step(c, p, r.dt, &r.opts, &stats);
    stepped = true;
  }
  // after a failed step p holds the last accepted Newton iterate: returned too
  if (stepped && r.p_out_host && status != RICH_ECUDA && status != RICH_ENONFINITE && status != RICH_ENOMEM)
    if (cudaMemcpyAsync(r.p_out_host, p, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess &&
        !status)
      status = RICH_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && !status) status = RICH_ECUDA;
  if (!se || !se->ctx) {  // one-off request, or a session whose creation failed part way
    dfree(p);
    if (c) rich_destroy(c);
  }
  q->res.status = status;
  q->res.stats = stats;
}

static void srv_worker(rich_server* s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreate(&st);  // a blocking stream: ordered with the legacy default stream
  for (;;) {
    SrvRequest* q = nullptr;
    SrvSession* se = nullptr;
    std::vector<SrvSession*> evict;
    std::vector<SrvRequest*> group;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      for (;;) {
        q = srv_pick(s, &evict);
        if (q || !evict.empty() || s->stop) break;
        s->cv_work.wait(lock);
      }
      if (q) {
        if (q->r.session) se = s->sessions[q->r.session];
        group.push_back(q);
        if (!se) srv_pick_mates(s, q, &group);
        const double t_admit = srv_now(s);
        for (SrvRequest* m : group) {
          ++s->in_flight;
          ++s->admitted;
          m->res.t_admit = t_admit;
          m->res.slot = slot;
          m->res.mem_estimate = m->est;
          m->res.mem_in_flight = s->reserved;
          m->res.batch_size = 1;
        }
        if (s->in_flight > s->max_in_flight) s->max_in_flight = s->in_flight;
      }
    }
    for (SrvSession* v : evict) srv_free_session(v, st);
    if (!q) {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->stop && s->queue.empty()) break;
      continue;
    }
    if (group.size() > 1) srv_run_batch(s, group, st);
    else srv_run(q, se, st);
    SrvSession* dead = nullptr;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (SrvRequest* m : group)
        if (!m->r.session) s->reserved -= m->est;
      if (se && !se->ctx) {  // the session's first request failed before creating its state
        s->sessions.erase(se->id);
        s->reserved -= se->est;
        dead = se;
        se = nullptr;
      }
      if (se) se->busy = false;
      const double t_done = srv_now(s);
      for (SrvRequest* m : group) {
        --s->in_flight;
        m->res.t_done = t_done;
        m->done = true;
      }
    }
    delete dead;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace rich

using namespace rich;

extern "C" {

void rich_default_server_opts(rich_server_opts* o) {
  if (!o) return;
  o->slots = 8;
  o->mem_budget_bytes = 0.0;
  o->max_sessions = 64;
  o->batch_max = 1;
  o->batch_min_cells = 300000;
}

int rich_server_create(const rich_server_opts* opts, rich_server** out) {
  if (!out) return RICH_EINVAL;
  *out = nullptr;
  rich_server_opts o;
  if (opts) o = *opts; else rich_default_server_opts(&o);
  if (o.slots < 1 || o.slots > 256 || o.max_sessions < 0 || o.batch_max < 1 || o.batch_max > 32) return RICH_EINVAL;
  rich_server* s = new rich_server();
  s->o = o;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaGetDevice");
    delete s;
    return RICH_ECUDA;
  }
  if (o.mem_budget_bytes > 0) {
    s->budget = o.mem_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    pool_trim();
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaMemGetInfo");
      delete s;
      return RICH_ECUDA;
    }
    s->budget = 0.8 * (double)fr;
  }
  for (int k = 0; k < o.slots; ++k) s->workers.emplace_back(srv_worker, s, k);
  *out = s;
  return RICH_OK;
}

int rich_server_submit(rich_server* s, const rich_request* req, long long* id_out) {
  if (!s || !req || !id_out) return RICH_EINVAL;
  const rich_request& r = *req;
  if (r.grid.nx < 1 || r.grid.ny < 1 || r.grid.nz < 1 || !(r.grid.lx > 0 && r.grid.ly > 0 && r.grid.lz > 0))
    return RICH_EINVAL;
  if (!(r.dt > 0) || !kmean_valid(r.kmean)) return RICH_EINVAL;
  if (r.precision != RICH_PREC_FP64 && r.precision != RICH_PREC_MIXED) return RICH_EINVAL;
  for (int f = 0; f < 6; ++f) {
    if (r.bc.kind[f] != RICH_BC_NOFLUX && r.bc.kind[f] != RICH_BC_DIRICHLET) return RICH_EINVAL;
    if (r.bc.value_field_dev[f]) return RICH_EINVAL;
  }
  if (r.session < 0 || (!r.p0_host && !r.session)) return RICH_EINVAL;
  SrvRequest* q = new SrvRequest();
  q->r = r;
  q->r.soil.ks_field_dev = nullptr;
  q->est = srv_estimate(r);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (q->est > s->budget) {
      delete q;
      return RICH_ELIMIT;
    }
    q->id = s->next_id++;
    q->res.t_submit = srv_now(s);
    s->reqs[q->id] = q;
    s->queue.push_back(q);
    *id_out = q->id;
  }
  s->cv_work.notify_one();
  return RICH_OK;
}

static int srv_take(rich_server* s, long long id, rich_request_result* out, bool block) {
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return RICH_EINVAL;
  SrvRequest* q = it->second;
  if (!q->done) {
    if (!block) return RICH_EBUSY;
    s->cv_done.wait(lock, [&] { return q->done; });
  }
  if (out) *out = q->res;
  s->reqs.erase(it);
  delete q;
  return RICH_OK;
}

int rich_server_poll(rich_server* s, long long id, rich_request_result* out) {
  if (!s) return RICH_EINVAL;
  return srv_take(s, id, out, false);
}

int rich_server_wait(rich_server* s, long long id, rich_request_result* out) {
  if (!s) return RICH_EINVAL;
  return srv_take(s, id, out, true);
}

int rich_server_drain(rich_server* s) {
  if (!s) return RICH_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  s->cv_done.wait(lock, [&] { return s->queue.empty() && s->in_flight == 0; });
  return RICH_OK;
}

int rich_server_counters(rich_server* s, long long* admitted, int* max_in_flight, double* reserved_bytes) {
  if (!s) return RICH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (admitted) *admitted = s->admitted;
  if (max_in_flight) *max_in_flight = s->max_in_flight;
  if (reserved_bytes) *reserved_bytes = s->reserved;
  return RICH_OK;
}

int rich_server_destroy(rich_server* s) {
  if (!s) return RICH_OK;
  rich_server_drain(s);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreate(&st);
  for (auto& kv : s->sessions) srv_free_session(kv.second, st);
  s->sessions.clear();
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return RICH_OK;
}

}  // extern "C"
