// Request server with continuous batching (include/jfft.h, jfft_server_*).
//
// Requests (grid, material field, load cases, tolerance, preconditioner, precision)
// are queued on submission. max_active worker threads, each with its own CUDA
// stream, take the first queued request that can be admitted now and solve it
// on a solver handle of its own; the streams let the GPU overlap the work of
// all running requests, and a request that arrives while others run starts as
// soon as a worker and the memory for its solver are free. Admission is by device
// memory: the workspace of every live solver (running or idle) counts against the
// budget; idle solvers of the right grid shape and precision are reused (their
// material, Poisson ratio, Jacobi scaling and Alg. 1 symbol are re-set), and idle
// solvers of other shapes are evicted, least recently used first, when a request
// needs their memory. Every solve is the same deterministic kernel sequence it
// would be alone, so a result does not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "jfft.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  jfft_grid grid = {};
  int kind = 0;
  double nu = 0.3, e_min = 0.0, e_max = 1.0, exponent = 1.0;
  std::vector<double> field, eps;
  int n_loads = 0;
  double tol = 0.0;
  int precond = 0, precision = 0, want_u = 0, max_loads = 0;
  size_t bytes = 0;
  // results
  std::vector<double> u, chom, rel;
  std::vector<int> iters, refine;
  int status = -1;
  int state = 0;  // 0 queued, 1 running, 2 done
  bool reused = false;
  Clock::time_point t_submit, t_start, t_end;
  std::string err;
};

struct ShapeKey {
  int d;
  int64_t n[3];
  int precision;
  int max_loads;
  bool operator<(const ShapeKey& o) const {
    if (d != o.d) return d < o.d;
    for (int a = 0; a < 3; ++a)
      if (n[a] != o.n[a]) return n[a] < o.n[a];
    if (precision != o.precision) return precision < o.precision;
    return max_loads < o.max_loads;
  }
  bool operator==(const ShapeKey& o) const { return !(*this < o) && !(o < *this); }
};

struct Idle {
  jfft_solver* h;
  ShapeKey key;
  size_t bytes;
  uint64_t last_use;
};

ShapeKey key_of(const Request& r) {
  ShapeKey k{};
  k.d = r.grid.dim;
  for (int a = 0; a < 3; ++a) k.n[a] = a < r.grid.dim ? r.grid.n[a] : 0;
  k.precision = r.precision;
  k.max_loads = r.max_loads;
  return k;
}

}  // namespace

struct jfft_server {
  jfft_server_options opt = {};
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<Idle> idle;
  size_t used = 0, peak_used = 0;
  uint64_t tick = 0;
  int64_t next_id = 1, submitted = 0, finished = 0, running = 0, creates = 0, reuses = 0, evictions = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;  // one per worker; outlive every solver that used them
  std::string err;
};

static double secs(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Under the lock: first queued request that can start now. Sets *solver to an idle
// solver of its shape (reuse) or reserves its bytes (create); appends evicted idle
// solvers to *evict. Returns nullptr if none can start.
static Request* pick(jfft_server* s, jfft_solver** solver, std::vector<jfft_solver*>* evict) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    Request* r = *it;
    const ShapeKey k = key_of(*r);
    for (size_t i = 0; i < s->idle.size(); ++i)
      if (s->idle[i].key == k) {
        *solver = s->idle[i].h;
        s->idle.erase(s->idle.begin() + i);
        s->queue.erase(it);
        r->reused = true;
        return r;
      }
    // free memory by evicting idle solvers of other shapes, least recently used first
    size_t avail = s->budget > s->used ? s->budget - s->used : 0;
    size_t evictable = 0;
    for (auto& e : s->idle) evictable += e.bytes;
    if (r->bytes > avail + evictable) continue;
    while (r->bytes > (s->budget > s->used ? s->budget - s->used : 0)) {
      auto lru = std::min_element(s->idle.begin(), s->idle.end(),
                                  [](const Idle& a, const Idle& b) { return a.last_use < b.last_use; });
      evict->push_back(lru->h);
      s->used -= lru->bytes;
      s->evictions++;
      s->idle.erase(lru);
    }
    s->used += r->bytes;
    s->peak_used = std::max(s->peak_used, s->used);
    *solver = nullptr;
    s->queue.erase(it);
    return r;
  }
  return nullptr;
}

static void run_request(jfft_server* s, Request* r, jfft_solver*& h, cudaStream_t st) {
  jfft_material mat;
  mat.kind = r->kind;
  mat.field = r->field.data();
  mat.nu = r->nu;
  mat.e_min = r->e_min;
  mat.e_max = r->e_max;
  mat.exponent = r->exponent;
  jfft_status rc;
  if (!h) {
    jfft_options o;
    jfft_default_options(&o);
    o.precision = r->precision;
    o.stream = st;
    o.max_loads = r->max_loads;
    o.device = s->opt.device;
    rc = jfft_create(&h, &r->grid, &mat, nullptr, &o);
    if (rc != JFFT_OK) {
      r->err = jfft_last_error(nullptr);
      h = nullptr;
    } else {
      std::lock_guard<std::mutex> lk(s->mu);
      s->creates++;
    }
  } else {
    rc = jfft_set_stream(h, st);
    if (rc == JFFT_OK) rc = jfft_set_material(h, &mat);
    if (rc != JFFT_OK) r->err = jfft_last_error(h);
    std::lock_guard<std::mutex> lk(s->mu);
    s->reuses++;
  }
  if (rc == JFFT_OK) {
    const int d = r->grid.dim, ds = d * (d + 1) / 2;
    int64_t N = 1;
    for (int a = 0; a < d; ++a) N *= r->grid.n[a];
    if (r->want_u) r->u.resize((size_t)r->n_loads * d * N);
    r->chom.resize((size_t)ds * r->n_loads);
    r->iters.resize(r->n_loads);
    r->rel.resize(r->n_loads);
    r->refine.resize(r->n_loads);
    jfft_result res = {};
    res.u = r->want_u ? r->u.data() : nullptr;
    res.stress = nullptr;
    res.C_hom = r->chom.data();
    res.iters = r->iters.data();
    res.rel_res = r->rel.data();
    res.refine_steps = r->refine.data();
    rc = jfft_solve(h, r->n_loads, r->eps.data(), r->tol, (jfft_precond)r->precond, &res);
    if (rc != JFFT_OK) r->err = jfft_last_error(h);
  }
  r->status = rc;
}

static void worker_main(jfft_server* s, cudaStream_t st) {
  cudaSetDevice(s->opt.device);
  for (;;) {
    Request* r = nullptr;
    jfft_solver* h = nullptr;
    std::vector<jfft_solver*> evict;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || (r = pick(s, &h, &evict)) != nullptr; });
      if (!r) break;
      r->state = 1;
      r->t_start = Clock::now();
      s->running++;
    }
    for (jfft_solver* e : evict) jfft_destroy(e);
    const bool created = h == nullptr;
    run_request(s, r, h, st);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_end = Clock::now();
      r->state = 2;
      s->running--;
      s->finished++;
      if (h) {
        s->idle.push_back(Idle{h, key_of(*r), r->bytes, ++s->tick});
      } else if (created) {
        s->used -= r->bytes;  // creation failed: release the reservation
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

extern "C" void jfft_server_default_options(jfft_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->max_active = 4;
  o->hbm_budget = 0;
  o->device = 0;
}

extern "C" jfft_status jfft_server_create(jfft_server** out, const jfft_server_options* opt) {
  if (!out) return JFFT_ERR_ARG;
  *out = nullptr;
  jfft_server_options o;
  jfft_server_default_options(&o);
  if (opt) o = *opt;
  if (o.max_active < 1 || o.max_active > 64) return JFFT_ERR_ARG;
  if (cudaSetDevice(o.device) != cudaSuccess) return JFFT_ERR_CUDA;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return JFFT_ERR_CUDA;
  jfft_server* s = new jfft_server();
  s->opt = o;
  s->budget = o.hbm_budget ? std::min(o.hbm_budget, fr) : (size_t)(0.8 * (double)fr);
  for (int i = 0; i < o.max_active; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
      delete s;
      return JFFT_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  for (int i = 0; i < o.max_active; ++i) s->workers.emplace_back(worker_main, s, s->streams[i]);
  *out = s;
  return JFFT_OK;
}

static jfft_status server_fail(jfft_server* s, jfft_status e, const char* m) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->err = m;
  return e;
}

extern "C" jfft_status jfft_server_submit(jfft_server* s, const jfft_request* q, int64_t* id_out) {
  if (!s || !q || !id_out) return JFFT_ERR_ARG;
  *id_out = 0;
  if (!q->material.field || !q->eps_bar || q->n_loads < 1)
    return server_fail(s, JFFT_ERR_ARG, "request needs a material field, strains and n_loads >= 1");
  const int d = q->grid.dim;
  const int ds = d * (d + 1) / 2;
  jfft_options o;
  jfft_default_options(&o);
  o.precision = q->precision;
  o.max_loads = d == 2 ? 3 : 6;
  if (q->n_loads > o.max_loads) return server_fail(s, JFFT_ERR_ARG, "n_loads exceeds the number of Mandel components");
  size_t bytes = 0;
  jfft_status e = jfft_workspace_estimate(&q->grid, &o, &bytes);
  if (e != JFFT_OK) return server_fail(s, e, "unsupported grid or precision");
  std::unique_ptr<Request> r(new Request());
  r->grid = q->grid;
  r->kind = q->material.kind;
  r->nu = q->material.nu;
  r->e_min = q->material.e_min;
  r->e_max = q->material.e_max;
  r->exponent = q->material.exponent;
  int64_t N = 1;
  for (int a = 0; a < d; ++a) N *= q->grid.n[a];
  r->field.assign(q->material.field, q->material.field + N);
  r->eps.assign(q->eps_bar, q->eps_bar + (size_t)q->n_loads * ds);
  r->n_loads = q->n_loads;
  r->tol = q->tol;
  r->precond = q->precond;
  r->precision = q->precision;
  r->want_u = q->want_u;
  r->max_loads = o.max_loads;
  r->bytes = bytes;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes > s->budget) {
    s->err = "request workspace exceeds the server's memory budget";
    return JFFT_ERR_OOM;
  }
  r->id = s->next_id++;
  *id_out = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->submitted++;
  s->cv_work.notify_one();
  return JFFT_OK;
}

extern "C" int jfft_server_poll(jfft_server* s, int64_t id) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  return it == s->reqs.end() ? -1 : it->second->state;
}

extern "C" jfft_status jfft_server_wait(jfft_server* s, int64_t id, jfft_result* res, double* timing) {
  if (!s) return JFFT_ERR_ARG;
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
      s->err = "unknown request id";
      return JFFT_ERR_ARG;
    }
    if (it->second->state == 0 && s->stop) {
      s->err = "the server stopped before the request started";
      return JFFT_ERR_ARG;
    }
    Request* p = it->second.get();
    s->cv_done.wait(lk, [&] { return p->state == 2; });
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (res) {
    if (res->u && !r->u.empty()) std::memcpy(res->u, r->u.data(), r->u.size() * sizeof(double));
    if (res->C_hom && !r->chom.empty()) std::memcpy(res->C_hom, r->chom.data(), r->chom.size() * sizeof(double));
    if (res->iters && !r->iters.empty()) std::memcpy(res->iters, r->iters.data(), r->iters.size() * sizeof(int));
    if (res->rel_res && !r->rel.empty()) std::memcpy(res->rel_res, r->rel.data(), r->rel.size() * sizeof(double));
    if (res->refine_steps && !r->refine.empty())
      std::memcpy(res->refine_steps, r->refine.data(), r->refine.size() * sizeof(int));
  }
  if (timing) {
    timing[0] = secs(r->t_submit, r->t_start);
    timing[1] = secs(r->t_start, r->t_end);
    timing[2] = secs(r->t_submit, r->t_end);
    timing[3] = r->reused ? 1.0 : 0.0;
  }
  if (r->status != JFFT_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = r->err;
  }
  return (jfft_status)r->status;
}

extern "C" jfft_status jfft_server_stats(jfft_server* s, jfft_server_counters* out) {
  if (!s || !out) return JFFT_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->finished = s->finished;
  out->queued = (int64_t)s->queue.size();
  out->running = s->running;
  out->budget = s->budget;
  out->used = s->used;
  out->peak_used = s->peak_used;
  out->solvers_created = s->creates;
  out->solvers_reused = s->reuses;
  out->solvers_evicted = s->evictions;
  return JFFT_OK;
}

extern "C" const char* jfft_server_last_error(jfft_server* s) {
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  thread_local std::string copy;
  copy = s->err;
  return copy.c_str();
}

extern "C" void jfft_server_destroy(jfft_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& e : s->idle) jfft_destroy(e.h);  // before the streams they last ran on
  for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
  delete s;
}
