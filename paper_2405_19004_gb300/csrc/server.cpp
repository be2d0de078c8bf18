// Continuous-batching server for Poisson solve requests.
//
// Requests (dimension, degree, level, sine-mode right-hand side) wait in a
// queue.  An engine thread admits them as solver slots and device memory
// (a fixed budget) become free: a slot is a vps handle whose level hierarchy
// stays resident and is reused by later requests of the same shape; idle
// slots are evicted, least recently used first, when memory is needed.
//
// Admitted requests of the same dimension, degree (and the server's
// precision) form a cohort that shares one CUDA stream.  Every request runs
// the preconditioned CG of the library as an asynchronous state machine
// whose V-cycles are run by the cohort: whenever no work of the cohort is in
// flight, the engine runs one V-cycle for every member that waits for one
// (cohort_vcycle: the colour passes, restrictions and prolongations of all
// members' levels as persistent kernels taking tiles from a device-side
// queue, one launch per step), then the rest of each member's CG iteration,
// and polls the members' events.  A request that arrives while others run
// joins its cohort at the next of these ticks; different cohorts run
// concurrently on their own streams.  A request's numbers depend only on its
// own data: every level of it goes through the same operations in the same
// order as alone, so its result is the same alone and in a mix.
//
// The engine never blocks on the GPU (it polls events); waits on the host
// side take a timeout.  No kernel waits on work it does not own: a
// persistent launch's queue is complete before the launch, so there is no
// device-side spin to bound.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "vps.h"
#include "vps_internal.h"

namespace {

double now_s() {
  using clock = std::chrono::steady_clock;
  static const clock::time_point t0 = clock::now();
  return std::chrono::duration<double>(clock::now() - t0).count();
}

struct Request {
  int64_t id = 0;
  int d = 0, k = 0, L = 0;
  std::vector<double> coef;
  std::vector<int> freq;
  double* x_out = nullptr;
  int64_t n = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = VPS_REQ_QUEUED;
  int status = VPS_OK;
  int iters = 0;
  double rel = 0;
};

struct Cohort;

enum SlotState { kCreating, kIdle, kActive, kCompleting, kFailed };

struct Slot {
  vps_context* h = nullptr;
  int d = 0, k = 0, L = 0;
  size_t bytes = 0;
  std::atomic<int> state{kCreating};  // written under mu; read by the engine without it
  int create_rc = VPS_OK;
  int64_t req = 0;  // the request of an active or completing slot
  double last_used = 0;
  Cohort* cohort = nullptr;
};

// Requests of one (dimension, degree): one stream, and the staging buffers
// of the batched V-cycles' queues (pinned host and device).
struct Cohort {
  int d = 0, k = 0;
  cudaStream_t stream = nullptr;
  void* q_host = nullptr;
  void* q_dev = nullptr;
  size_t q_cap = 0;
};

constexpr size_t kCohortQueueBytes = size_t(4) << 20;
constexpr int kMaxModesPrepared = 8;   // sine modes the slots' buffers are sized for
constexpr int kMaxCreating = 4;        // hierarchies being built at a time

// A job of the provisioning thread: build a slot's hierarchy, or destroy an
// evicted one.
struct ProvJob {
  Slot* create = nullptr;
  vps_context* destroy = nullptr;
};

// A job of the completion thread: copy a finished request's result from the
// slot's pinned staging into the caller's buffer.
struct DoneJob {
  Slot* slot = nullptr;
  int64_t req = 0;
  const double* x = nullptr;
  int state = 0, status = 0, iters = 0;
  double rel = 0.0;
};

}  // namespace

// Three host threads: the engine (admission, cohort V-cycles, polling; it
// never waits for the GPU or for an allocation), the provisioner (builds and
// destroys hierarchies: vps_create allocates and uploads, vps_destroy
// synchronises) and the completer (copies results into the callers' buffers).
struct vps_server_ctx {
  size_t budget = 0;
  int max_active = 1;
  int precision = VPS_FP32;
  double rtol = 1e-10;
  int max_it = 100;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // request state changes, slot readiness
  std::condition_variable prov_cv;  // provisioner jobs
  std::condition_variable done_cv;  // completer jobs
  std::thread engine, provisioner, completer;
  std::atomic<bool> stop{false};
  std::map<int64_t, Request> reqs;
  std::deque<int64_t> queue;
  std::vector<std::unique_ptr<Slot>> slots;      // vector: engine thread; Slot fields: under mu
  std::vector<std::unique_ptr<Cohort>> cohorts;  // engine thread only
  std::deque<ProvJob> prov_jobs;                 // under mu
  std::deque<DoneJob> done_jobs;                 // under mu
  size_t used = 0;          // engine thread only (budget accounting)
  // batching statistics (under mu)
  int64_t ticks = 0, batched_launches = 0;
  int max_per_launch = 0, max_per_tick = 0;
  // host time of the engine's parts and of the helper threads (under mu)
  double t_admit = 0, t_tick = 0, t_poll = 0, t_create = 0, t_copy = 0;
  int64_t next_id = 1;
  int64_t n_done = 0;
  int active = 0;
  std::string err;

  void run();
  void run_provisioner();
  void run_completer();
  bool admit();
  bool tick(Cohort& c);
  Cohort* cohort_of(int d, int k, int* rc);
  void fail_request(int64_t id, int status);
  void finish_error(Slot& s, int status, int iters, double rel);
  void release();
};

namespace {

double since(double t0) { return now_s() - t0; }

}  // namespace

// The cohort of (d, k), created on first use.
Cohort* vps_server_ctx::cohort_of(int d, int k, int* rc) {
  *rc = VPS_OK;
  for (auto& c : cohorts)
    if (c->d == d && c->k == k) return c.get();
  auto c = std::make_unique<Cohort>();
  c->d = d;
  c->k = k;
  c->q_cap = kCohortQueueBytes;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&c->q_host, c->q_cap);
  if (e == cudaSuccess) e = cudaMalloc(&c->q_dev, c->q_cap);
  if (e != cudaSuccess) {
    if (c->q_dev) cudaFree(c->q_dev);
    if (c->q_host) cudaFreeHost(c->q_host);
    if (c->stream) cudaStreamDestroy(c->stream);
    std::lock_guard<std::mutex> lock(mu);
    err = cudaGetErrorString(e);
    *rc = e == cudaErrorMemoryAllocation ? VPS_ENOMEM : VPS_ECUDA;
    return nullptr;
  }
  cohorts.push_back(std::move(c));
  return cohorts.back().get();
}

// Runs one V-cycle for every active member of c that waits for one, then
// the rest of their CG iterations, if none of the cohort's work is in flight.
bool vps_server_ctx::tick(Cohort& c) {
  std::vector<Slot*> pending;
  for (auto& sp : slots) {
    Slot& s = *sp;
    if (s.state != kActive || s.cohort != &c) continue;
    if (vps::cg_async_pending_vcycle(s.h)) pending.push_back(&s);
    else return false;  // a member's work is still in flight
  }
  if (pending.empty()) return false;
  const double t0 = now_s();
  std::vector<vps_context*> hs;
  for (Slot* s : pending) hs.push_back(s->h);
  int64_t launches = 0;
  int per_launch = 0;
  int rc = vps::cohort_vcycle(hs.data(), (int)hs.size(), c.q_host, c.q_dev, c.q_cap, &launches,
                              &per_launch);
  for (Slot* s : pending) {
    int r = rc ? rc : vps::cg_async_resume(s->h);
    if (r) {
      {
        std::lock_guard<std::mutex> lock(mu);
        err = vps::handle_error(rc ? hs[0] : s->h);
      }
      finish_error(*s, r, 0, 0.0);
    }
  }
  std::lock_guard<std::mutex> lock(mu);
  ++ticks;
  batched_launches += launches;
  max_per_launch = std::max(max_per_launch, per_launch);
  max_per_tick = std::max(max_per_tick, (int)hs.size());
  t_tick += since(t0);
  return true;
}

// Marks a queued request failed (engine thread, not holding mu).
void vps_server_ctx::fail_request(int64_t id, int status) {
  std::lock_guard<std::mutex> lock(mu);
  auto q = std::find(queue.begin(), queue.end(), id);
  if (q != queue.end()) queue.erase(q);
  Request& r = reqs[id];
  r.state = VPS_REQ_FAILED;
  r.status = status;
  r.t_done = now_s();
  ++n_done;
  cv.notify_all();
}

// Ends the request of an active slot with an error (no result to copy).
void vps_server_ctx::finish_error(Slot& s, int status, int iters, double rel) {
  std::lock_guard<std::mutex> lock(mu);
  Request& r = reqs[s.req];
  r.state = VPS_REQ_FAILED;
  r.status = status;
  r.iters = iters;
  r.rel = rel;
  r.t_done = now_s();
  s.req = 0;
  s.state = kIdle;
  s.last_used = r.t_done;
  --active;
  ++n_done;
  cv.notify_all();
}

// Admission: starts queued requests that have an idle slot of their shape
// (queue order, within the first 64), and orders new hierarchies from the
// provisioner for shapes with more waiting requests than idle or building
// slots.  Returns true if anything changed.
bool vps_server_ctx::admit() {
  const double t0 = now_s();
  bool changed = false;
  // slots whose creation failed: fail one waiting request of their shape
  for (auto it = slots.begin(); it != slots.end();) {
    int st, rc;
    {
      std::lock_guard<std::mutex> lock(mu);
      st = (*it)->state;
      rc = (*it)->create_rc;
    }
    if (st != kFailed) {
      ++it;
      continue;
    }
    const Slot& s = **it;
    int64_t victim = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      for (int64_t id : queue) {
        const Request& r = reqs[id];
        if (r.d == s.d && r.k == s.k && r.L == s.L) {
          victim = id;
          break;
        }
      }
    }
    if (victim) fail_request(victim, rc);
    used -= s.bytes;
    it = slots.erase(it);
    changed = true;
  }
  // start requests with an idle slot
  std::vector<std::pair<int64_t, Slot*>> starts;
  std::vector<Request> snaps;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (size_t qi = 0; qi < queue.size() && qi < 64 && active < max_active;) {
      const Request& r = reqs[queue[qi]];
      Slot* slot = nullptr;
      for (auto& s : slots)
        if (s->state == kIdle && s->d == r.d && s->k == r.k && s->L == r.L) {
          slot = s.get();
          break;
        }
      if (!slot) {
        ++qi;
        continue;
      }
      const int64_t id = queue[qi];
      queue.erase(queue.begin() + qi);
      Request& rr = reqs[id];
      rr.state = VPS_REQ_RUNNING;
      rr.t_start = now_s();
      ++active;
      slot->state = kActive;
      slot->req = id;
      starts.push_back({id, slot});
      snaps.push_back(rr);
    }
  }
  for (size_t i = 0; i < starts.size(); ++i) {
    Slot* slot = starts[i].second;
    const Request& r = snaps[i];
    const int rc = vps::cg_async_begin(slot->h, (int)r.coef.size(), r.coef.data(), r.freq.data(),
                                       rtol, max_it);
    if (rc) {
      {
        std::lock_guard<std::mutex> lock(mu);
        err = vps::handle_error(slot->h);
      }
      finish_error(*slot, rc, 0, 0.0);
    }
    changed = true;
  }
  // order hierarchies for waiting requests without a slot
  std::vector<Request> want;
  {
    std::lock_guard<std::mutex> lock(mu);
    int creating = 0;
    for (auto& s : slots) creating += s->state == kCreating;
    std::map<std::tuple<int, int, int>, int> spare;  // idle or building slots per shape
    for (auto& s : slots)
      if (s->state == kIdle || s->state == kCreating) ++spare[std::make_tuple(s->d, s->k, s->L)];
    for (size_t qi = 0; qi < queue.size() && qi < 64 && creating < kMaxCreating; ++qi) {
      const Request& r = reqs[queue[qi]];
      int& sp = spare[std::make_tuple(r.d, r.k, r.L)];
      if (sp > 0) {
        --sp;
        continue;
      }
      want.push_back(r);
      ++creating;
    }
  }
  for (const Request& r : want) {
    const size_t need = vps::estimate_device_bytes(r.d, r.k, r.L, precision);
    if (need > budget) {  // can never fit
      fail_request(r.id, VPS_ENOMEM);
      changed = true;
      continue;
    }
    // evict idle slots, least recently used first, until the request fits
    bool fits = true;
    while (used + need > budget) {
      auto victim = slots.end();
      {
        std::lock_guard<std::mutex> lock(mu);
        for (auto it = slots.begin(); it != slots.end(); ++it)
          if ((*it)->state == kIdle &&
              (victim == slots.end() || (*it)->last_used < (*victim)->last_used))
            victim = it;
      }
      if (victim == slots.end()) {
        fits = false;  // wait for a running request to finish
        break;
      }
      used -= (*victim)->bytes;
      {
        std::lock_guard<std::mutex> lock(mu);
        prov_jobs.push_back({nullptr, (*victim)->h});
        prov_cv.notify_one();
      }
      slots.erase(victim);
      changed = true;
    }
    if (!fits) break;
    int rc = VPS_OK;
    Cohort* c = cohort_of(r.d, r.k, &rc);
    if (rc) {
      fail_request(r.id, rc);
      changed = true;
      continue;
    }
    auto s = std::make_unique<Slot>();
    s->d = r.d;
    s->k = r.k;
    s->L = r.L;
    s->cohort = c;
    s->bytes = need;
    used += need;
    std::lock_guard<std::mutex> lock(mu);
    prov_jobs.push_back({s.get(), nullptr});
    prov_cv.notify_one();
    slots.push_back(std::move(s));
    changed = true;
  }
  std::lock_guard<std::mutex> lock(mu);
  t_admit += since(t0);
  return changed;
}

void vps_server_ctx::run_provisioner() {
  cudaSetDevice(device);
  while (true) {
    ProvJob job;
    {
      std::unique_lock<std::mutex> lock(mu);
      prov_cv.wait(lock, [&] { return stop.load() || !prov_jobs.empty(); });
      if (prov_jobs.empty()) return;  // stopping
      job = prov_jobs.front();
      prov_jobs.pop_front();
    }
    const double t0 = now_s();
    if (job.destroy) {
      vps_destroy(job.destroy);
    } else if (Slot* s = job.create) {
      vps_context* h = nullptr;
      int rc = vps_create(s->d, s->k, s->L, precision, VPS_MULTIPLICATIVE, 1.0, 1, 1,
                          s->cohort->stream, &h);
      if (!rc) {
        vps::set_external_vcycle(h, true);
        rc = vps::cg_async_prepare(h, kMaxModesPrepared);
      }
      std::lock_guard<std::mutex> lock(mu);
      if (rc) {
        err = h ? vps::handle_error(h) : vps_last_error(nullptr);
        if (h) vps_destroy(h);
        s->create_rc = rc;
        s->state = kFailed;
      } else {
        s->h = h;
        s->state = kIdle;
      }
      cv.notify_all();
    }
    std::lock_guard<std::mutex> lock(mu);
    t_create += since(t0);
  }
}

void vps_server_ctx::run_completer() {
  while (true) {
    DoneJob job;
    {
      std::unique_lock<std::mutex> lock(mu);
      done_cv.wait(lock, [&] { return stop.load() || !done_jobs.empty(); });
      if (done_jobs.empty()) return;  // stopping
      job = done_jobs.front();
      done_jobs.pop_front();
    }
    const double t0 = now_s();
    double* out = nullptr;
    int64_t n = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      const Request& r = reqs[job.req];
      out = r.x_out;
      n = r.n;
    }
    if (out && job.x) std::memcpy(out, job.x, (size_t)n * sizeof(double));
    std::lock_guard<std::mutex> lock(mu);
    Request& r = reqs[job.req];
    r.state = job.state;
    r.status = job.status;
    r.iters = job.iters;
    r.rel = job.rel;
    r.t_done = now_s();
    job.slot->req = 0;
    job.slot->state = kIdle;
    job.slot->last_used = r.t_done;
    --active;
    ++n_done;
    t_copy += since(t0);
    cv.notify_all();
  }
}

void vps_server_ctx::run() {
  cudaSetDevice(device);
  while (!stop.load()) {
    bool progressed = false;
    const double t0 = now_s();
    for (auto& sp : slots) {
      Slot& s = *sp;
      if (s.state != kActive || vps::cg_async_pending_vcycle(s.h)) continue;
      int done = 0, status = 0, iters = 0;
      double rel = 0;
      const double* x = nullptr;
      const int rc = vps::cg_async_poll(s.h, &done, &status, &iters, &rel, &x);
      if (rc) {
        {
          std::lock_guard<std::mutex> lock(mu);
          err = vps::handle_error(s.h);
        }
        finish_error(s, rc, iters, rel);
        progressed = true;
      } else if (done) {
        std::lock_guard<std::mutex> lock(mu);
        s.state = kCompleting;
        done_jobs.push_back({&s, s.req, x, status == VPS_OK ? VPS_REQ_DONE : VPS_REQ_FAILED,
                             status, iters, rel});
        done_cv.notify_one();
        progressed = true;
      } else if (vps::cg_async_pending_vcycle(s.h)) {
        progressed = true;
      }
    }
    {
      std::lock_guard<std::mutex> lock(mu);
      t_poll += since(t0);
    }
    if (admit()) progressed = true;
    for (auto& c : cohorts)
      if (tick(*c)) progressed = true;
    if (!progressed) {
      std::unique_lock<std::mutex> lock(mu);
      if (queue.empty() && active == 0)
        cv.wait_for(lock, std::chrono::milliseconds(2));
      else
        cv.wait_for(lock, std::chrono::microseconds(20));
    }
  }
}

// Stops the helper threads and frees the slots and the cohorts (after the
// engine has stopped).
void vps_server_ctx::release() {
  {
    std::lock_guard<std::mutex> lock(mu);
    prov_cv.notify_all();
    done_cv.notify_all();
  }
  if (provisioner.joinable()) provisioner.join();
  if (completer.joinable()) completer.join();
  for (auto& c : cohorts)
    if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& sl : slots)
    if (sl->h) vps_destroy(sl->h);
  slots.clear();
  for (auto& c : cohorts) {
    if (c->q_dev) cudaFree(c->q_dev);
    if (c->q_host) cudaFreeHost(c->q_host);
    if (c->stream) cudaStreamDestroy(c->stream);
  }
  cohorts.clear();
}

extern "C" {

int vps_server_create(size_t memory_budget, int max_active, int precision, double rtol,
                      int max_it, vps_server* out) {
  if (!out) return VPS_EINVAL;
  *out = nullptr;
  if (memory_budget == 0 || max_active < 1 || max_active > 1024 ||
      (precision != VPS_FP32 && precision != VPS_FP64) || !(rtol > 0.0) || max_it < 1) {
    vps::set_thread_error("vps_server_create: invalid argument");
    return VPS_EINVAL;
  }
  auto* s = new vps_server_ctx();
  s->budget = memory_budget;
  s->max_active = max_active;
  s->precision = precision;
  s->rtol = rtol;
  s->max_it = max_it;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    vps::set_thread_error("vps_server_create: no CUDA device");
    return VPS_ECUDA;
  }
  s->engine = std::thread([s] { s->run(); });
  s->provisioner = std::thread([s] { s->run_provisioner(); });
  s->completer = std::thread([s] { s->run_completer(); });
  *out = s;
  return VPS_OK;
}

int vps_server_submit(vps_server s, int dim, int degree, int level, int n_modes,
                      const double* coef, const int* freq, double* x_out, int64_t* id) {
  if (!s || !id || n_modes < 1 || n_modes > 4096 || !coef || !freq || (dim != 2 && dim != 3) ||
      degree < 1 || degree > VPS_MAX_DEGREE || level < 1 || level > 24)
    return VPS_EINVAL;
  // the same size limit as vps_create (checked in floating point, before
  // any product below can overflow)
  if (!(vps::level_elements(dim, degree, level) <= 2147483647.0)) return VPS_EINVAL;
  Request r;
  r.d = dim;
  r.k = degree;
  r.L = level;
  r.coef.assign(coef, coef + n_modes);
  r.freq.assign(freq, freq + n_modes * dim);
  r.x_out = x_out;
  const int64_t ni = (int64_t)degree * (1 << level) - 1;
  r.n = dim == 3 ? ni * ni * ni : ni * ni;
  std::lock_guard<std::mutex> lock(s->mu);
  r.id = s->next_id++;
  r.t_submit = now_s();
  *id = r.id;
  s->reqs[r.id] = std::move(r);
  s->queue.push_back(*id);
  s->cv.notify_all();
  return VPS_OK;
}

int vps_server_query(vps_server s, int64_t id, int* state, int* status, int* iters,
                     double* rel_res, double* queue_s, double* latency_s) {
  if (!s) return VPS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return VPS_EINVAL;
  const Request& r = it->second;
  if (state) *state = r.state;
  if (status) *status = r.status;
  if (iters) *iters = r.iters;
  if (rel_res) *rel_res = r.rel;
  const bool started = r.state != VPS_REQ_QUEUED;
  const bool ended = r.state == VPS_REQ_DONE || r.state == VPS_REQ_FAILED;
  if (queue_s) *queue_s = started ? r.t_start - r.t_submit : -1.0;
  if (latency_s) *latency_s = ended ? r.t_done - r.t_submit : -1.0;
  return VPS_OK;
}

int vps_server_wait(vps_server s, int64_t id, double timeout_s) {
  if (!s) return VPS_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto ready = [&] {
    if (id == 0) return s->n_done == s->next_id - 1;
    auto it = s->reqs.find(id);
    return it == s->reqs.end() || it->second.state == VPS_REQ_DONE ||
           it->second.state == VPS_REQ_FAILED;
  };
  if (!s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)) return VPS_ETIMEOUT;
  return VPS_OK;
}

int vps_server_stats(vps_server s, int64_t* submitted, int64_t* done, int* active, int* queued) {
  if (!s) return VPS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (submitted) *submitted = s->next_id - 1;
  if (done) *done = s->n_done;
  if (active) *active = s->active;
  if (queued) *queued = (int)s->queue.size();
  return VPS_OK;
}

const char* vps_server_last_error(vps_server s) { return s ? s->err.c_str() : ""; }

int vps_server_batch_stats(vps_server s, int64_t* ticks, int64_t* batched_launches,
                           int* max_requests_per_launch, int* max_requests_per_tick) {
  if (!s) return VPS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (ticks) *ticks = s->ticks;
  if (batched_launches) *batched_launches = s->batched_launches;
  if (max_requests_per_launch) *max_requests_per_launch = s->max_per_launch;
  if (max_requests_per_tick) *max_requests_per_tick = s->max_per_tick;
  return VPS_OK;
}

int vps_server_host_times(vps_server s, double* seconds) {
  if (!s || !seconds) return VPS_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  seconds[0] = s->t_admit;
  seconds[1] = s->t_tick;
  seconds[2] = s->t_poll;
  seconds[3] = s->t_create;
  seconds[4] = s->t_copy;
  return VPS_OK;
}

int vps_server_destroy(vps_server s) {
  if (!s) return VPS_OK;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->engine.joinable()) s->engine.join();
  s->release();
  delete s;
  return VPS_OK;
}

}  // extern "C"
