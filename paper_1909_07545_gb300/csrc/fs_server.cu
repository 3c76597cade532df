// fs_server.cu -- continuous-batching request server over many rigs (the
// contract is in fs_server.h).
//
// One dispatcher thread owns every device call.  Requests wait in one FIFO;
// the dispatcher scans it in arrival order and starts each request whose
// rig is idle, whose rig has no earlier request still waiting, for which a
// slot is free, and whose rig state is resident or can be made resident
// within the memory budget (evicting idle rigs, least recently used first).
// A started request runs on its rig's stream: host-to-device copies of the
// pair, one fs_solve (a replayed CUDA graph: the rig's planes are fixed, so
// the graph's pointers never change), device-to-host copies of the result,
// then a host callback that stamps the completion time and wakes the
// dispatcher and any waiter.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "fs.h"
#include "fs_server.h"
#include "fs_stages.h"

extern fs_status fs_internal_set_error(fs_status s, const char* msg);
extern fs_status fs_internal_validate(const fs_calib cam[2], const fs_pose* pose, int W, int H,
                                      int levels, const fs_params* prm);
extern cudaError_t fs_internal_malloc(void** p, size_t bytes, const char* site);

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

fs_status set_error(fs_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
fs_status set_error(fs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return fs_internal_set_error(s, buf);
}

struct Rig {
  fs_calib cam[2];
  fs_pose pose;
  fs_params prm;
  int W = 0, H = 0, levels = 0;
  size_t bytes = 0;               // device bytes while resident
  fs_handle* h = nullptr;         // resident state (null: not resident)
  float* planes = nullptr;        // I0, I1, disparity (also the warm start), depth
  cudaStream_t stream = nullptr;
  bool has_prev = false;          // planes hold the previous frame's disparity
  bool busy = false;              // a request of this rig is in flight
  unsigned long long last_use = 0;
  size_t n() const { return (size_t)W * H; }
};

struct Request;

}  // namespace

struct fs_server {
  fs_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // dispatcher: queue or slots changed
  std::condition_variable cv_done;   // waiters: some request completed
  std::vector<Rig*> rigs;
  std::deque<Request*> pending;      // arrival order
  std::unordered_map<long long, Request*> known;   // submitted, not yet waited for
  long long next_id = 1;
  int inflight = 0;
  size_t resident = 0, peak = 0;
  unsigned long long tick = 0;
  bool stop = false;
  std::thread worker;
  // statistics since the last reset
  std::vector<double> lat;
  long long submitted = 0, completed = 0, failed = 0, cold = 0, evictions = 0, cancelled = 0;
  bool have_first = false;
  Clock::time_point first_submit, last_done;
};

namespace {

struct Request {
  fs_server* srv = nullptr;
  long long id = 0;
  int rig = 0;
  const float* I0 = nullptr;
  const float* I1 = nullptr;
  float* disp = nullptr;
  float* depth = nullptr;
  Clock::time_point t_submit, t_done;
  bool done = false;
  bool waited = false;            // a thread is in fs_server_wait for it
  fs_status status = FS_OK;
  std::string msg;
};

// Host callback on the rig's stream after the result's copies: stamps the
// completion and releases the rig and the slot.  No CUDA calls here.
void CUDART_CB on_request_done(void* arg) {
  Request* r = (Request*)arg;
  fs_server* s = r->srv;
  Clock::time_point t = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->t_done = t;
    r->done = true;
    s->rigs[r->rig]->busy = false;
    --s->inflight;
    ++s->completed;
    if (r->status != FS_OK) ++s->failed;
    s->lat.push_back(ms_between(r->t_submit, t));
    s->last_done = t;
  }
  s->cv_work.notify_one();
  s->cv_done.notify_all();
}

// A rig's device state taken out of the rig (under the lock) so that it can
// be freed with the lock released: fs_destroy / cudaFree may wait for the
// device, and the completion callbacks of other rigs need the lock.
struct Detached {
  fs_handle* h = nullptr;
  float* planes = nullptr;
  cudaStream_t stream = nullptr;
};

Detached detach_rig_state(fs_server* s, Rig* rg) {
  Detached d{rg->h, rg->planes, rg->stream};
  if (rg->h) s->resident -= rg->bytes;
  rg->h = nullptr;
  rg->planes = nullptr;
  rg->has_prev = false;
  return d;
}

void destroy_detached(const Detached& d) {
  if (!d.h) return;
  cudaStreamSynchronize(d.stream);
  fs_destroy(d.h);
  if (d.planes) cudaFree(d.planes);
}

// Make rig state resident (called without the lock; the rig is marked busy
// so nothing else touches it).  Returns FS_OK or the error of fs_create /
// the plane allocation, with *msg set.
fs_status make_resident(fs_server* s, Rig* rg, std::string* msg) {
  fs_params p = rg->prm;
  p.use_graph = 1;
  fs_status st = fs_create(rg->cam, &rg->pose, rg->W, rg->H, rg->levels, &p, rg->stream, &rg->h);
  if (st != FS_OK) {
    *msg = fs_last_error();
    rg->h = nullptr;
    return st;
  }
  cudaError_t e = fs_internal_malloc((void**)&rg->planes, 4 * rg->n() * sizeof(float), "planes");
  if (e != cudaSuccess) {
    fs_destroy(rg->h);
    rg->h = nullptr;
    rg->planes = nullptr;
    *msg = std::string("rig plane allocation failed: ") + cudaGetErrorString(e);
    return FS_ENOMEM;
  }
  if (s->cfg.autotune && (st = fs_autotune(rg->h, s->cfg.iters, nullptr)) != FS_OK) {
    *msg = fs_last_error();
    fs_destroy(rg->h);
    cudaFree(rg->planes);
    rg->h = nullptr;
    rg->planes = nullptr;
    return st;
  }
  return FS_OK;
}

// Enqueue one admitted request on its rig's stream (no lock held).
fs_status enqueue_request(fs_server* s, Rig* rg, Request* r, bool cold_start, std::string* msg) {
  const size_t n = rg->n(), bytes = n * sizeof(float);
  float* dI0 = rg->planes;
  float* dI1 = rg->planes + n;
  float* dD = rg->planes + 2 * n;
  float* dZ = rg->planes + 3 * n;
  cudaStream_t st = rg->stream;
  cudaError_t e = cudaMemcpyAsync(dI0, r->I0, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dI1, r->I1, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    *msg = std::string("input copy failed: ") + cudaGetErrorString(e);
    return FS_ECUDA;
  }
  // a warm start from the disparity reads the previous one from dD and
  // writes the new one over it (the library copies d_init in before anything
  // writes d_disp); a continued one reads the handle's own u and w
  fs_status st_solve;
  if (cold_start)
    st_solve = fs_solve(rg->h, dI0, dI1, nullptr, s->cfg.cold_warps, s->cfg.cold_iters, dD, dZ);
  else if (s->cfg.warm_mode == 1)
    st_solve = fs_solve_continue(rg->h, dI0, dI1, s->cfg.warps, s->cfg.iters, dD, dZ);
  else
    st_solve = fs_solve(rg->h, dI0, dI1, dD, s->cfg.warps, s->cfg.iters, dD, dZ);
  if (st_solve != FS_OK) {
    *msg = fs_last_error();
    return st_solve;
  }
  if (r->disp) e = cudaMemcpyAsync(r->disp, dD, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && r->depth) e = cudaMemcpyAsync(r->depth, dZ, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_request_done, r);
  if (e != cudaSuccess) {
    *msg = std::string("result copy failed: ") + cudaGetErrorString(e);
    return FS_ECUDA;
  }
  return FS_OK;
}

// Fail a request on the dispatcher thread without device work.
void fail_request(fs_server* s, Request* r, fs_status st, const std::string& msg) {
  Clock::time_point t = Clock::now();
  r->status = st;
  r->msg = msg;
  r->t_done = t;
  r->done = true;
  ++s->completed;
  ++s->failed;
  s->lat.push_back(ms_between(r->t_submit, t));
  s->last_done = t;
}

// One admission pass (lock held on entry and exit).  Returns true if it
// started or failed a request, i.e. the queue changed.
bool admit_one(fs_server* s, std::unique_lock<std::mutex>& lk) {
  std::vector<char> blocked(s->rigs.size(), 0);   // rigs with an earlier waiting request
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    if (s->inflight >= s->cfg.max_inflight) return false;
    Request* r = *it;
    Rig* rg = s->rigs[r->rig];
    if (rg->busy || blocked[r->rig]) { blocked[r->rig] = 1; continue; }
    std::vector<Detached> evicted;
    if (!rg->h) {
      // evict idle rigs, least recently used first, until this one fits;
      // decide first, so that nothing is evicted for a rig that still
      // would not fit
      std::vector<Rig*> victims;
      size_t res = s->resident;
      while (res + rg->bytes > s->cfg.hbm_budget) {
        Rig* victim = nullptr;
        for (Rig* o : s->rigs)
          if (o->h && !o->busy && std::find(victims.begin(), victims.end(), o) == victims.end() &&
              (!victim || o->last_use < victim->last_use))
            victim = o;
        if (!victim) break;
        victims.push_back(victim);
        res -= victim->bytes;
      }
      if (res + rg->bytes > s->cfg.hbm_budget) { blocked[r->rig] = 1; continue; }
      for (Rig* v : victims) {
        evicted.push_back(detach_rig_state(s, v));
        ++s->evictions;
      }
    }
    // start it
    s->pending.erase(it);
    rg->busy = true;
    ++s->inflight;
    rg->last_use = ++s->tick;
    const bool need_state = rg->h == nullptr;
    if (need_state) s->resident += rg->bytes;   // reserved before the allocation
    s->peak = std::max(s->peak, s->resident);
    const bool cold_start = need_state || !rg->has_prev;
    if (cold_start) ++s->cold;
    lk.unlock();
    for (const Detached& d : evicted) destroy_detached(d);
    std::string msg;
    fs_status st = FS_OK;
    if (need_state && (st = make_resident(s, rg, &msg)) != FS_OK) {
      lk.lock();
      s->resident -= rg->bytes;
      rg->busy = false;
      --s->inflight;
      fail_request(s, r, st, msg);
      s->cv_done.notify_all();
      return true;
    }
    st = enqueue_request(s, rg, r, cold_start, &msg);
    lk.lock();
    if (st != FS_OK) {
      rg->busy = false;
      --s->inflight;
      rg->has_prev = false;
      fail_request(s, r, st, msg);
      s->cv_done.notify_all();
    } else {
      rg->has_prev = true;
    }
    return true;
  }
  return false;
}

void dispatcher(fs_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    if (admit_one(s, lk)) continue;
    s->cv_work.wait(lk);
  }
}

fs_status check_server(const fs_server* s) {
  if (!s) return set_error(FS_EINVAL, "null server");
  return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs_server_default_config(fs_server_config* out) {
  if (!out) return set_error(FS_EINVAL, "null config");
  memset(out, 0, sizeof(*out));
  out->hbm_budget = (size_t)40 << 30;
  out->max_inflight = 2;
  out->warps = 3;
  out->iters = 50;
  out->cold_warps = 10;
  out->cold_iters = 100;
  out->warm_mode = 1;
  out->autotune = 1;
  return FS_OK;
}

fs_status fs_server_create(const fs_server_config* cfg, fs_server** out) {
  if (!out) return set_error(FS_EINVAL, "null output server pointer");
  *out = nullptr;
  fs_server_config c;
  if (cfg) {
    c = *cfg;
    if (c.hbm_budget == 0) c.hbm_budget = (size_t)40 << 30;
  } else {
    fs_server_default_config(&c);
  }
  if (c.max_inflight < 1) return set_error(FS_EINVAL, "max_inflight must be >= 1");
  if (c.warps < 1 || c.iters < 1 || c.cold_warps < 1 || c.cold_iters < 1)
    return set_error(FS_EINVAL, "warps and iters must be >= 1");
  if (c.warm_mode != 0 && c.warm_mode != 1) return set_error(FS_EINVAL, "warm_mode must be 0 or 1");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FS_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  // never plan for more than the device has free now (less 1 GiB of headroom
  // for the CUDA context, graphs and the callers' own buffers)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
    const size_t headroom = (size_t)1 << 30;
    const size_t avail = free_b > headroom ? free_b - headroom : 0;
    if (c.hbm_budget > avail) c.hbm_budget = avail;
  }
  fs_server* s = new (std::nothrow) fs_server();
  if (!s) return set_error(FS_ENOMEM, "host allocation failed");
  s->cfg = c;
  s->device = dev;
  s->worker = std::thread(dispatcher, s);
  *out = s;
  return FS_OK;
}

fs_status fs_server_add_rig(fs_server* s, const fs_calib cam[2], const fs_pose* pose, int W,
                            int H, int levels, const fs_params* prm, int* rig_id) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  if (!cam || !pose || !rig_id) return set_error(FS_EINVAL, "null argument");
  fs_params p;
  if (prm) p = *prm; else fs_default_params(&p);
  // fs_create's checks now; the handle itself is made when the rig's first
  // request is admitted
  if ((st = fs_internal_validate(cam, pose, W, H, levels, &p)) != FS_OK) return st;
  size_t bytes = 0;
  if ((st = fs_state_bytes(W, H, levels, &p, &bytes)) != FS_OK) return st;
  bytes += 4 * (size_t)W * H * sizeof(float);
  if (bytes > s->cfg.hbm_budget)
    return set_error(FS_ENOMEM, "rig state of %zu bytes exceeds the budget of %zu", bytes,
                     s->cfg.hbm_budget);
  Rig* rg = new (std::nothrow) Rig();
  if (!rg) return set_error(FS_ENOMEM, "host allocation failed");
  rg->cam[0] = cam[0];
  rg->cam[1] = cam[1];
  rg->pose = *pose;
  rg->prm = p;
  rg->W = W;
  rg->H = H;
  rg->levels = levels;
  rg->bytes = bytes;
  cudaError_t e = cudaStreamCreateWithFlags(&rg->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete rg;
    return set_error(FS_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> g(s->mu);
  *rig_id = (int)s->rigs.size();
  s->rigs.push_back(rg);
  return FS_OK;
}

fs_status fs_server_submit(fs_server* s, int rig, const float* h_I0, const float* h_I1,
                           float* h_disp, float* h_depth, long long* req_id) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  if (!h_I0 || !h_I1 || !req_id) return set_error(FS_EINVAL, "null argument");
  Request* r = new (std::nothrow) Request();
  if (!r) return set_error(FS_ENOMEM, "host allocation failed");
  r->srv = s;
  r->rig = rig;
  r->I0 = h_I0;
  r->I1 = h_I1;
  r->disp = h_disp;
  r->depth = h_depth;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (rig < 0 || rig >= (int)s->rigs.size()) {
      delete r;
      return set_error(FS_EINVAL, "unknown rig %d", rig);
    }
    r->id = s->next_id++;
    s->pending.push_back(r);
    s->known[r->id] = r;
    ++s->submitted;
    if (!s->have_first) { s->first_submit = r->t_submit; s->have_first = true; }
    *req_id = r->id;
  }
  s->cv_work.notify_one();
  return FS_OK;
}

fs_status fs_server_wait(fs_server* s, long long req_id, double timeout_s, double* latency_ms) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->known.find(req_id);
  if (it == s->known.end()) return set_error(FS_EINVAL, "unknown request %lld", req_id);
  Request* r = it->second;
  // one waiter per request: the one that sees it done deletes it
  if (r->waited) return set_error(FS_EINVAL, "request %lld is already being waited for", req_id);
  r->waited = true;
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    r->waited = false;
    return set_error(FS_ETIMEOUT, "request %lld still pending", req_id);
  }
  if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
  st = r->status;
  std::string msg = r->msg;
  // by key: a submission while this thread slept may have rehashed the map
  // and invalidated the iterator found above
  s->known.erase(req_id);
  delete r;
  lk.unlock();
  if (st != FS_OK) return set_error(st, "request %lld: %s", req_id, msg.c_str());
  return FS_OK;
}

fs_status fs_server_cancel(fs_server* s, long long req_id) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  std::lock_guard<std::mutex> g(s->mu);
  auto kit = s->known.find(req_id);
  if (kit == s->known.end()) return set_error(FS_EINVAL, "unknown request %lld", req_id);
  auto it = std::find(s->pending.begin(), s->pending.end(), kit->second);
  if (it == s->pending.end())
    return set_error(FS_EINVAL, "request %lld is already on the GPU or done", req_id);
  Request* r = *it;
  s->pending.erase(it);
  r->status = FS_ECANCELLED;
  r->msg = "cancelled before it ran";
  r->t_done = Clock::now();
  r->done = true;
  ++s->cancelled;
  s->cv_done.notify_all();
  s->cv_work.notify_one();
  return FS_OK;
}

fs_status fs_server_drain(fs_server* s, double timeout_s) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->pending.empty() && s->inflight == 0; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, idle);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) {
    return set_error(FS_ETIMEOUT, "%zu queued and %d in flight", s->pending.size(), s->inflight);
  }
  return FS_OK;
}

fs_status fs_server_stats_read(fs_server* s, fs_server_stats* out, int reset) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  if (!out) return set_error(FS_EINVAL, "null output");
  std::lock_guard<std::mutex> g(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->cold = s->cold;
  out->evictions = s->evictions;
  out->cancelled = s->cancelled;
  out->resident_bytes = s->resident;
  out->peak_resident_bytes = s->peak;
  if (!s->lat.empty()) {
    std::vector<double> v = s->lat;
    std::sort(v.begin(), v.end());
    // nearest-rank percentiles
    auto pct = [&](double q) {
      size_t k = (size_t)std::ceil(q / 100.0 * v.size());
      return v[k == 0 ? 0 : k - 1];
    };
    out->p50_ms = pct(50.0);
    out->p99_ms = pct(99.0);
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / v.size();
    double span = ms_between(s->first_submit, s->last_done);
    out->frames_per_s = span > 0 ? 1000.0 * v.size() / span : 0.0;
  }
  if (reset) {
    s->lat.clear();
    s->submitted = s->completed = s->failed = s->cold = s->evictions = s->cancelled = 0;
    s->have_first = false;
    s->peak = s->resident;
  }
  return FS_OK;
}

fs_status fs_server_evict_all(fs_server* s) {
  fs_status st;
  if ((st = check_server(s)) != FS_OK) return st;
  std::vector<Detached> ds;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->inflight == 0; });
    for (Rig* rg : s->rigs) ds.push_back(detach_rig_state(s, rg));
  }
  for (const Detached& d : ds) destroy_detached(d);
  return FS_OK;
}

fs_status fs_server_destroy(fs_server* s) {
  if (!s) return FS_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending.clear();
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->inflight == 0; });
  }
  for (Rig* rg : s->rigs) {
    destroy_detached(detach_rig_state(s, rg));
    if (rg->stream) cudaStreamDestroy(rg->stream);
    delete rg;
  }
  for (auto& kv : s->known) delete kv.second;
  delete s;
  return FS_OK;
}

}  // extern "C"
