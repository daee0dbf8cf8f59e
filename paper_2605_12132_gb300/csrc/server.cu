// Continuous-batching request server for field-advance and envelope-advance requests (no counterpart
// in the paper).  See include/fdetd.h for the contract of the fdetd_server_* calls.
//
// One scheduler thread owns every device resource of the admitted requests.  Each round it
//   1. admits queued requests first-come first-served while their device footprint fits the HBM budget
//      (a request that does not fit waits; nothing overtakes it);
//   2. hands admitted requests to plan-builder threads (the FP64 eigen-solve of a field plan runs on the
//      host), which also allocate the device state and copy the inputs in on the request's own stream;
//   3. advances every ready field request together: they are the instances of one batch (one captured
//      CUDA graph per step: a persistent grouped projection and back-projection launch per tensor-core
//      precision, every instance's spectral kernel on its own branch), re-captured whenever a request
//      joins or leaves, replayed for a chunk of steps no longer than the shortest remaining request;
//   4. advances every ready envelope request by its own chunk on its own stream, concurrently with the
//      field batch;
//   5. retires finished requests: copies the result to the caller's host buffer, frees the device state
//      and the plan, returns the bytes to the budget, stamps the completion time.
// A request that fails (plan construction, allocation, a device timeout) ends in the failed state with
// its message; its bytes return to the budget and the server keeps running.  In dry-run mode no CUDA
// call is made: plan building checks the request's sizes on the host and a chunk takes a fixed host
// time per step, so the scheduling logic runs on machines without a GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fdetd.h"
#include "kernels.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
  uint64_t id = 0;
  fdetd_request req;
  std::vector<int> modes;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = FDETD_TICKET_QUEUED;
  int err = FDETD_OK;
  std::string msg;
  // owned by the builder until `built`, then by the scheduler
  bool built = false;
  fdetd_plan_t plan = nullptr;
  envelope_plan_t eplan = nullptr;
  void* d_state = nullptr;
  void* d_aux = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  int done_steps = 0;
  int chunk = 0;
};

size_t pad_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct fdetd_server_s {
  size_t budget = 0, used = 0, peak = 0;
  int chunk_steps = 16;
  bool dry = false;
  double dry_step_s = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_build;
  std::deque<Ticket*> queue;                 // submitted, not admitted
  std::deque<Ticket*> build_jobs;            // admitted, waiting for a builder
  std::vector<Ticket*> building;             // admitted, plan under construction
  std::vector<Ticket*> fields, envelopes;    // on the device
  std::unordered_map<uint64_t, Ticket*> all;
  uint64_t next_id = 1;
  bool stop = false;            // no more submissions; the scheduler drains and exits
  bool builders_stop = false;   // set once the scheduler has exited
  std::thread sched;
  std::vector<std::thread> builders;
  // field batch
  fdetd_batch_t batch = nullptr;
  bool batch_dirty = true;
  cudaStream_t bstream = nullptr;
  cudaEvent_t bevent = nullptr;
  // statistics
  uint64_t completed = 0, failed = 0, recaptures = 0, rounds = 0;
  double served_cell_steps = 0;
};

// ---------------------------------------------------------------- footprint
extern "C" size_t fdetd_request_device_bytes(const fdetd_request* r) {
  if (!r) return 0;
  const size_t Nz = (size_t)std::max(r->Nz, 0), n = (size_t)std::max(r->Nr, 0);
  if (r->kind == FDETD_REQUEST_ENVELOPE) {
    const size_t plane = Nz * n;
    // state (a, a~) c64 and chi f32; plan: three Taylor buffers of (a, a~), chi + sigma^2, radial band
    return plane * 16 + plane * 4 + plane * 48 + plane * 4 + n * (size_t)(r->order + 2) * 4 + 4096;
  }
  const size_t nm = (size_t)std::max(r->nmodes, 0);
  const bool fp64 = r->precision == FDETD_PREC_FP64;
  const size_t elt = fp64 ? 16 : 8, cells = nm * Nz * n;
  size_t b = cells * 6 * elt + (r->J ? cells * 3 * elt : 0);              // resident fields and current
  b += cells * 9 * elt;                                                    // coefficient scratch
  if (Nz > 4096 || (fp64 && Nz > 2048)) b += nm * 2 * 3 * n * Nz * elt;   // source term of the two-kernel path
  b += nm * 2 * n * Nz * (fp64 ? 32 : 16) + nm * 2 * n * 16;              // phase and eigenvalue tables
  b += Nz * 16 + Nz * 32 + 2 * (Nz + 64) * elt + 64;                        // z symbols, twiddles, flag
  if (r->precision == FDETD_PREC_BF16X3 || r->precision == FDETD_PREC_BF16X6) {
    const size_t np = r->precision == FDETD_PREC_BF16X3 ? 2 : 3;
    const size_t nks = (n + 31) / 32, njb = (n + 255) / 256 * 2, ksb = (n + 63) / 64, nrb = (n + 127) / 128;
    b += nm * 2 * np * 9 * nks * njb * 8192 + nm * 2 * np * 9 * ksb * nrb * 16384;   // pre-tiled P, Q pieces
    b += nm * np * 6 * ksb * (pad_up(Nz, 64) / 64) * 16384;                           // split coefficients
    b += 2 * 1024 * 1024;                                                               // tile tables
  } else {
    b += 2 * nm * 2 * (3 * n) * (3 * n) * (fp64 ? 8 : 4);                  // P and Q
  }
  return b + b / 64 + 4096;
}

// ---------------------------------------------------------------- builders
static void release_device(Ticket* t) {
  if (t->plan) fdetd_plan_destroy(t->plan);
  if (t->eplan) envelope_plan_destroy(t->eplan);
  if (t->d_state) cudaFree(t->d_state);
  if (t->d_aux) cudaFree(t->d_aux);
  if (t->event) cudaEventDestroy(t->event);
  if (t->stream) cudaStreamDestroy(t->stream);
  t->plan = nullptr;
  t->eplan = nullptr;
  t->d_state = t->d_aux = nullptr;
  t->event = nullptr;
  t->stream = nullptr;
}

static int build_one(fdetd_server_s* s, Ticket* t, std::string& msg) {
  const fdetd_request& r = t->req;
  if (s->dry) {
    // the host-side checks a plan makes before any device work
    if (r.order < 2 || r.order > 32 || (r.order & 1) || r.Nr < r.order / 2 + 1 || r.Nz < 2) {
      msg = "request sizes rejected by the plan";
      return FDETD_ERR_ARG;
    }
    return FDETD_OK;
  }
  char buf[512];
  int rc;
  if (r.kind == FDETD_REQUEST_ENVELOPE)
    rc = envelope_plan(&t->eplan, r.Nz, r.Nr, r.order, r.taylor_order, r.dz, r.dr, r.dt, r.k0);
  else
    rc = fdetd_plan_modes(&t->plan, r.Nz, r.Nr, t->modes.data(), r.nmodes, r.order, r.dz, r.dr, r.dt, r.precision, 0);
  if (rc) {
    fdetd_last_error(buf, sizeof(buf));
    msg = std::string("plan: ") + buf;
    return rc;
  }
  const size_t plane = (size_t)r.Nz * r.Nr;
  cudaError_t e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->event, cudaEventDisableTiming);
  if (r.kind == FDETD_REQUEST_ENVELOPE) {
    if (e == cudaSuccess) e = cudaMalloc(&t->d_state, 2 * plane * 8);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_aux, plane * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_state, r.fields, 2 * plane * 8, cudaMemcpyHostToDevice, t->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_aux, r.chi, plane * 4, cudaMemcpyHostToDevice, t->stream);
  } else {
    const size_t elt = r.precision == FDETD_PREC_FP64 ? 16 : 8;
    const size_t fb = (size_t)r.nmodes * 6 * plane * elt, jb = (size_t)r.nmodes * 3 * plane * elt;
    if (e == cudaSuccess) e = cudaMalloc(&t->d_state, fb);
    if (e == cudaSuccess && r.J) e = cudaMalloc(&t->d_aux, jb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_state, r.fields, fb, cudaMemcpyHostToDevice, t->stream);
    if (e == cudaSuccess && r.J) e = cudaMemcpyAsync(t->d_aux, r.J, jb, cudaMemcpyHostToDevice, t->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    msg = std::string("request state: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FDETD_ERR_OOM : FDETD_ERR_CUDA;
  }
  return FDETD_OK;
}

static void builder_loop(fdetd_server_s* s) {
  for (;;) {
    Ticket* t = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_build.wait(lk, [&] { return s->builders_stop || !s->build_jobs.empty(); });
      if (s->build_jobs.empty()) return;
      t = s->build_jobs.front();
      s->build_jobs.pop_front();
    }
    std::string msg;
    const int rc = build_one(s, t, msg);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      t->err = rc;
      t->msg = msg;
      t->built = true;
    }
    s->cv_sched.notify_one();
  }
}

// ---------------------------------------------------------------- scheduler
static void finish(fdetd_server_s* s, Ticket* t, int rc, const std::string& msg) {
  // called by the scheduler with the lock NOT held; device release first
  if (!s->dry) release_device(t);
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= t->bytes;
  t->t_done = now_s();
  if (rc == FDETD_OK) {
    t->state = FDETD_TICKET_DONE;
    ++s->completed;
    const double modes = t->req.kind == FDETD_REQUEST_ENVELOPE ? 1.0 : (double)t->req.nmodes;
    s->served_cell_steps += (double)t->req.Nz * t->req.Nr * modes * t->req.steps;
  } else {
    t->state = FDETD_TICKET_FAILED;
    t->err = rc;
    t->msg = msg;
    ++s->failed;
  }
  s->cv_done.notify_all();
}

static int rebuild_batch(fdetd_server_s* s) {
  if (s->batch) fdetd_batch_destroy(s->batch);
  s->batch = nullptr;
  if (s->fields.empty()) return FDETD_OK;
  int rc = fdetd_batch_create(&s->batch);
  if (!rc) rc = fdetd_batch_set_autotune(s->batch, 0);
  for (Ticket* t : s->fields)
    if (!rc) rc = fdetd_batch_add(s->batch, t->plan, t->d_state, t->d_aux, nullptr);
  if (!rc) rc = fdetd_batch_capture(s->batch, 1, s->bstream);
  ++s->recaptures;
  return rc;
}

static void retire_field(fdetd_server_s* s, Ticket* t) {
  const fdetd_request& r = t->req;
  int rc = FDETD_OK;
  std::string msg;
  if (!s->dry) {
    rc = fdetd_plan_status(t->plan, t->stream);
    if (rc) {
      char buf[512];
      fdetd_last_error(buf, sizeof(buf));
      msg = buf;
    } else if (r.out) {
      const size_t elt = r.precision == FDETD_PREC_FP64 ? 16 : 8;
      const size_t fb = (size_t)r.nmodes * 6 * r.Nz * r.Nr * elt;
      cudaError_t e = cudaMemcpyAsync(r.out, t->d_state, fb, cudaMemcpyDeviceToHost, t->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
      if (e != cudaSuccess) {
        rc = FDETD_ERR_CUDA;
        msg = cudaGetErrorString(e);
      }
    }
  }
  finish(s, t, rc, msg);
}

static void retire_envelope(fdetd_server_s* s, Ticket* t) {
  const fdetd_request& r = t->req;
  int rc = FDETD_OK;
  std::string msg;
  if (!s->dry && r.out) {
    cudaError_t e = cudaMemcpyAsync(r.out, t->d_state, (size_t)2 * r.Nz * r.Nr * 8, cudaMemcpyDeviceToHost, t->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
    if (e != cudaSuccess) {
      rc = FDETD_ERR_CUDA;
      msg = cudaGetErrorString(e);
    }
  }
  finish(s, t, rc, msg);
}

static void sched_loop(fdetd_server_s* s) {
  if (!s->dry) {
    cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s->bevent, cudaEventDisableTiming);
  }
  for (;;) {
    std::vector<Ticket*> ready, broken;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // 1. admission, first come first served under the budget
      while (!s->queue.empty() && s->used + s->queue.front()->bytes <= s->budget) {
        Ticket* t = s->queue.front();
        s->queue.pop_front();
        s->used += t->bytes;
        s->peak = std::max(s->peak, s->used);
        t->state = FDETD_TICKET_ADMITTED;
        t->t_admit = now_s();
        s->build_jobs.push_back(t);
        s->building.push_back(t);
      }
      s->cv_build.notify_all();
      // 2. built plans join the device set
      std::vector<Ticket*> still;
      for (Ticket* t : s->building) {
        if (!t->built) {
          still.push_back(t);
          continue;
        }
        (t->err ? broken : ready).push_back(t);
      }
      s->building.swap(still);
      if (s->stop && s->queue.empty() && s->building.empty() && s->fields.empty() && s->envelopes.empty() &&
          ready.empty() && broken.empty())
        break;
      if (ready.empty() && broken.empty() && s->fields.empty() && s->envelopes.empty()) {
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      for (Ticket* t : ready) t->state = FDETD_TICKET_RUNNING;
    }
    for (Ticket* t : broken) finish(s, t, t->err, t->msg);
    for (Ticket* t : ready) {
      if (t->req.kind == FDETD_REQUEST_ENVELOPE) {
        s->envelopes.push_back(t);
      } else {
        s->fields.push_back(t);
        s->batch_dirty = true;
      }
    }
    ++s->rounds;
    // 3. the field batch: one chunk no longer than the shortest remaining request
    int fchunk = 0;
    if (!s->fields.empty()) {
      fchunk = s->chunk_steps;
      for (Ticket* t : s->fields) fchunk = std::min(fchunk, t->req.steps - t->done_steps);
      if (!s->dry) {
        int rc = FDETD_OK;
        if (s->batch_dirty) rc = rebuild_batch(s);
        s->batch_dirty = false;
        for (int k = 0; k < fchunk && rc == FDETD_OK; ++k) rc = fdetd_batch_launch(s->batch, s->bstream);
        if (rc == FDETD_OK && cudaEventRecord(s->bevent, s->bstream) != cudaSuccess) rc = FDETD_ERR_CUDA;
        if (rc != FDETD_OK) {
          char buf[512];
          fdetd_last_error(buf, sizeof(buf));
          for (Ticket* t : s->fields) finish(s, t, rc, std::string("batch: ") + buf);
          s->fields.clear();
          s->batch_dirty = true;
          fchunk = 0;
        }
      }
    }
    // 4. envelope requests, each on its own stream, concurrently with the field batch
    for (Ticket* t : s->envelopes) {
      t->chunk = std::min(s->chunk_steps, t->req.steps - t->done_steps);
      if (!s->dry) {
        int rc = envelope_step(t->eplan, t->d_state, (const float*)t->d_aux, t->chunk, t->stream);
        if (rc == FDETD_OK && cudaEventRecord(t->event, t->stream) != cudaSuccess) rc = FDETD_ERR_CUDA;
        if (rc != FDETD_OK) t->chunk = -rc;  // marks the failure for the retirement pass
      }
    }
    if (s->dry) {
      int longest = fchunk;
      for (Ticket* t : s->envelopes) longest = std::max(longest, t->chunk);
      std::this_thread::sleep_for(std::chrono::duration<double>(s->dry_step_s * longest));
    } else {
      if (fchunk > 0) cudaEventSynchronize(s->bevent);
      for (Ticket* t : s->envelopes)
        if (t->chunk > 0) cudaEventSynchronize(t->event);
    }
    // 5. retire what finished
    std::vector<Ticket*> keep;
    for (Ticket* t : s->fields) {
      t->done_steps += fchunk;
      if (t->done_steps >= t->req.steps) {
        retire_field(s, t);
        s->batch_dirty = true;
      } else {
        keep.push_back(t);
      }
    }
    s->fields.swap(keep);
    keep.clear();
    for (Ticket* t : s->envelopes) {
      if (t->chunk < 0) {
        finish(s, t, -t->chunk, "envelope step failed");
        continue;
      }
      t->done_steps += t->chunk;
      if (t->done_steps >= t->req.steps)
        retire_envelope(s, t);
      else
        keep.push_back(t);
    }
    s->envelopes.swap(keep);
  }
  if (s->batch) fdetd_batch_destroy(s->batch);
  s->batch = nullptr;
  if (s->bevent) cudaEventDestroy(s->bevent);
  if (s->bstream) cudaStreamDestroy(s->bstream);
}

// ---------------------------------------------------------------- C ABI
extern "C" int fdetd_server_create(fdetd_server_t* out, size_t hbm_budget_bytes, int chunk_steps, int plan_threads,
                                   uint64_t flags) {
  if (!out) return fdetd::set_error(FDETD_ERR_ARG, "out is null");
  *out = nullptr;
  if (!hbm_budget_bytes || chunk_steps < 1 || plan_threads < 1 || plan_threads > 64)
    return fdetd::set_error(FDETD_ERR_ARG, "budget, chunk_steps and plan_threads (1..64) must be positive");
  fdetd_server_s* s = new fdetd_server_s();
  s->budget = hbm_budget_bytes;
  s->chunk_steps = chunk_steps;
  s->dry = (flags & FDETD_SERVER_DRY_RUN) != 0;
  s->dry_step_s = s->dry ? 1e-4 : 0.0;
  if (!s->dry) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      delete s;
      return fdetd::set_error(FDETD_ERR_CUDA, "no CUDA device");
    }
  }
  for (int i = 0; i < plan_threads; ++i) s->builders.emplace_back(builder_loop, s);
  s->sched = std::thread(sched_loop, s);
  *out = s;
  return FDETD_OK;
}

extern "C" int fdetd_server_submit(fdetd_server_t s, const fdetd_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return fdetd::set_error(FDETD_ERR_ARG, "null argument");
  if (r->kind != FDETD_REQUEST_FIELD && r->kind != FDETD_REQUEST_ENVELOPE)
    return fdetd::set_error(FDETD_ERR_ARG, "unknown request kind");
  if (r->Nz < 1 || r->Nr < 1 || r->steps < 1 || !r->fields)
    return fdetd::set_error(FDETD_ERR_ARG, "request needs positive sizes and steps and its input state");
  if (r->kind == FDETD_REQUEST_FIELD && (r->nmodes < 1 || r->nmodes > 64 || !r->modes))
    return fdetd::set_error(FDETD_ERR_ARG, "field request needs 1..64 modes");
  if (r->kind == FDETD_REQUEST_ENVELOPE && !r->chi)
    return fdetd::set_error(FDETD_ERR_ARG, "envelope request needs chi");
  Ticket* t = new Ticket();
  t->req = *r;
  if (r->kind == FDETD_REQUEST_FIELD) t->modes.assign(r->modes, r->modes + r->nmodes);
  t->req.modes = nullptr;
  t->bytes = fdetd_request_device_bytes(r);
  t->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete t;
      return fdetd::set_error(FDETD_ERR_ARG, "server is shutting down");
    }
    if (t->bytes > s->budget) {
      const size_t need = t->bytes;
      delete t;
      return fdetd::set_error(FDETD_ERR_OOM, "request needs " + std::to_string(need) +
                                                 " device bytes, more than the whole budget");
    }
    t->id = s->next_id++;
    s->all[t->id] = t;
    s->queue.push_back(t);
    *ticket = t->id;
  }
  s->cv_sched.notify_one();
  return FDETD_OK;
}

static int ticket_info(fdetd_server_s* s, uint64_t id, int* state, double* latency_s) {
  auto it = s->all.find(id);
  if (it == s->all.end()) return fdetd::set_error(FDETD_ERR_ARG, "unknown ticket");
  Ticket* t = it->second;
  if (state) *state = t->state;
  if (latency_s) *latency_s = t->state >= FDETD_TICKET_DONE ? t->t_done - t->t_submit : -1.0;
  if (t->state == FDETD_TICKET_FAILED) return fdetd::set_error(t->err, "request failed: " + t->msg);
  return FDETD_OK;
}

extern "C" int fdetd_server_poll(fdetd_server_t s, uint64_t ticket, int* state, double* latency_s) {
  if (!s) return fdetd::set_error(FDETD_ERR_ARG, "server is null");
  std::lock_guard<std::mutex> lk(s->mu);
  return ticket_info(s, ticket, state, latency_s);
}

extern "C" int fdetd_server_wait(fdetd_server_t s, uint64_t ticket, double timeout_s, double* latency_s) {
  if (!s) return fdetd::set_error(FDETD_ERR_ARG, "server is null");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fdetd::set_error(FDETD_ERR_ARG, "unknown ticket");
  Ticket* t = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(timeout_s, 0.0));
  s->cv_done.wait_until(lk, until, [&] { return t->state >= FDETD_TICKET_DONE; });
  if (t->state < FDETD_TICKET_DONE) return fdetd::set_error(FDETD_ERR_TIMEOUT, "request not finished in time");
  return ticket_info(s, ticket, nullptr, latency_s);
}

extern "C" int fdetd_server_ticket_times(fdetd_server_t s, uint64_t ticket, double* times) {
  if (!s || !times) return fdetd::set_error(FDETD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fdetd::set_error(FDETD_ERR_ARG, "unknown ticket");
  times[0] = it->second->t_submit;
  times[1] = it->second->t_admit;
  times[2] = it->second->t_done;
  return FDETD_OK;
}

extern "C" int fdetd_server_stats(fdetd_server_t s, fdetd_server_stats_t* st) {
  if (!s || !st) return fdetd::set_error(FDETD_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->budget_bytes = s->budget;
  st->used_bytes = s->used;
  st->peak_bytes = s->peak;
  st->queued = s->queue.size();
  st->building = s->building.size();
  st->running = 0;
  for (auto& kv : s->all)
    if (kv.second->state == FDETD_TICKET_RUNNING) ++st->running;
  st->completed = s->completed;
  st->failed = s->failed;
  st->recaptures = s->recaptures;
  st->rounds = s->rounds;
  st->served_cell_steps = s->served_cell_steps;
  return FDETD_OK;
}

extern "C" int fdetd_server_cancel_queued(fdetd_server_t s, uint64_t* cancelled) {
  if (!s) return fdetd::set_error(FDETD_ERR_ARG, "server is null");
  uint64_t n = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (Ticket* q : s->queue) {
      q->state = FDETD_TICKET_FAILED;
      q->err = FDETD_ERR_ARG;
      q->msg = "cancelled before admission";
      q->t_done = t;
      ++s->failed;
      ++n;
    }
    s->queue.clear();
  }
  s->cv_done.notify_all();
  if (cancelled) *cancelled = n;
  return FDETD_OK;
}

extern "C" int fdetd_server_destroy(fdetd_server_t s) {
  if (!s) return FDETD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  s->cv_build.notify_all();
  if (s->sched.joinable()) s->sched.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->builders_stop = true;
  }
  s->cv_build.notify_all();
  for (auto& b : s->builders)
    if (b.joinable()) b.join();
  for (auto& kv : s->all) delete kv.second;
  delete s;
  return FDETD_OK;
}
