// Batched stepping and the serving runtime (host code around the step kernels).
//
// A batch advances many independent simulations with one CUDA-graph launch per step: the
// step of every member is captured on its own branch stream, the branches are joined into one
// graph, and the instantiated graph is replayed.  Kernels of different members overlap on the
// GPU, which is what lets many small grids fill the GPU's SMs.  The reference-map buffers of a grid
// alternate between two parities, so a batch keeps two graphs (even and odd steps) per
// membership.
//
// The server admits simulation jobs under a device-memory budget (each job's footprint is the
// exact byte count its grid will request), keeps their fields resident, steps all running jobs
// together through a batch, and records submit / admit / completion times.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "rmt.h"
#include "rmt_internal.h"

void rmt_count_launches(long n);

struct rmt_batch {
  cudaStream_t s = nullptr;    // launch stream (the caller's)
  cudaStream_t cap = nullptr;  // origin stream of the captures
  cudaEvent_t fork = nullptr;
  std::vector<rmt_grid*> g;
  std::vector<cudaStream_t> bs;  // one branch stream per member
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long nodes[2] = {0, 0};
  std::vector<int> par0;  // members' parities when exec[0] was captured
  int phase = 0;          // which of the two graphs runs next
  long captures = 0;      // graphs captured and instantiated
  double capture_s = 0;   // host time spent on them
  char msg[256] = {0};
};

namespace {

rmt_status bfail(rmt_batch* b, rmt_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->msg, sizeof b->msg, fmt, ap);
  va_end(ap);
  return st;
}

#define BCK(b, call)                                                                           \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, RMT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void drop(rmt_batch* b) {
  for (int p = 0; p < 2; p++) {
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
    b->exec[p] = nullptr;
    b->nodes[p] = 0;
  }
  b->par0.clear();
  b->phase = 0;
}

// one graph: every member's step on its branch, forked from and joined into the origin stream
rmt_status capture(rmt_batch* b, int ph) {
  const auto t0 = std::chrono::steady_clock::now();
  const long c0 = rmt_kernel_launches();
  BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  rmt_status st = RMT_OK;
  rmt_grid* failed = nullptr;
  // fork: every branch starts after the origin's (empty) head; join: the origin waits for all
  // branches only after the last one has been recorded, so the branches stay independent
  if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) st = RMT_ECUDA;
  for (size_t i = 0; i < b->g.size() && st == RMT_OK; i++) {
    if (cudaStreamWaitEvent(b->bs[i], b->fork, 0) != cudaSuccess) {
      st = RMT_ECUDA;
      break;
    }
    st = grid_capture_step(b->g[i], b->bs[i]);
    if (st != RMT_OK) failed = b->g[i];
    if (st == RMT_OK && cudaEventRecord(b->join[i], b->bs[i]) != cudaSuccess) st = RMT_ECUDA;
  }
  for (size_t i = 0; i < b->g.size() && st == RMT_OK; i++)
    if (cudaStreamWaitEvent(b->cap, b->join[i], 0) != cudaSuccess) st = RMT_ECUDA;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  const long nodes = rmt_kernel_launches() - c0;
  rmt_count_launches(-nodes);  // counted per replay
  if (st != RMT_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, st != RMT_OK ? st : RMT_ECUDA, "batch capture failed (%s)",
                 st != RMT_OK ? (failed ? rmt_last_error(failed) : "fork/join") : cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec[ph], graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return bfail(b, RMT_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
  b->nodes[ph] = nodes;
  b->captures++;
  b->capture_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return RMT_OK;
}

}  // namespace

extern "C" {

rmt_status rmt_batch_create(void* stream, rmt_batch** out) {
  if (!out) return RMT_EINVAL;
  *out = nullptr;
  rmt_batch* b = new (std::nothrow) rmt_batch();
  if (!b) return RMT_ENOMEM;
  b->s = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    rmt_batch_destroy(b);
    return RMT_ECUDA;
  }
  *out = b;
  return RMT_OK;
}

rmt_status rmt_batch_add(rmt_batch* b, rmt_grid* g) {
  if (!b || !g) return RMT_EINVAL;
  if (std::find(b->g.begin(), b->g.end(), g) != b->g.end()) return bfail(b, RMT_EINVAL, "already a member");
  BCK(b, cudaStreamSynchronize(b->s));
  rmt_status st = grid_join_batch(g, b->s);
  if (st != RMT_OK) return bfail(b, st, "member rejected: %s", rmt_last_error(g));
  cudaStream_t bs = nullptr;
  cudaEvent_t ev = nullptr;
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    if (bs) cudaStreamDestroy(bs);
    grid_leave_batch(g);
    return bfail(b, RMT_ECUDA, "stream/event creation failed");
  }
  b->g.push_back(g);
  b->bs.push_back(bs);
  b->join.push_back(ev);
  drop(b);
  return RMT_OK;
}

rmt_status rmt_batch_remove(rmt_batch* b, rmt_grid* g) {
  if (!b || !g) return RMT_EINVAL;
  auto it = std::find(b->g.begin(), b->g.end(), g);
  if (it == b->g.end()) return bfail(b, RMT_EINVAL, "not a member");
  BCK(b, cudaStreamSynchronize(b->s));
  const size_t i = it - b->g.begin();
  cudaStreamDestroy(b->bs[i]);
  cudaEventDestroy(b->join[i]);
  b->g.erase(b->g.begin() + i);
  b->bs.erase(b->bs.begin() + i);
  b->join.erase(b->join.begin() + i);
  grid_leave_batch(g);
  drop(b);
  return RMT_OK;
}

rmt_status rmt_batch_step(rmt_batch* b, int nsteps) {
  if (!b || nsteps < 0) return RMT_EINVAL;
  if (b->g.empty()) return RMT_OK;
  for (int k = 0; k < nsteps; k++) {
    // the graphs hold each member's buffers of one parity: recapture if a member moved on
    bool stale = b->par0.size() != b->g.size();
    for (size_t i = 0; !stale && i < b->g.size(); i++) stale = grid_parity(b->g[i]) != (b->par0[i] ^ b->phase);
    if (stale) {
      drop(b);
      for (rmt_grid* m : b->g) b->par0.push_back(grid_parity(m));
    }
    const int ph = b->phase;
    if (!b->exec[ph]) {
      rmt_status st = capture(b, ph);
      if (st != RMT_OK) return st;
    }
    for (rmt_grid* m : b->g) {
      const rmt_status st = grid_pre_step(m, b->s);
      if (st != RMT_OK) return bfail(b, st, "member: %s", rmt_last_error(m));
    }
    BCK(b, cudaGraphLaunch(b->exec[ph], b->s));
    rmt_count_launches(b->nodes[ph]);
    for (rmt_grid* m : b->g) grid_advance_host(m);
    b->phase ^= 1;
  }
  return RMT_OK;
}

rmt_status rmt_batch_sync(rmt_batch* b) {
  if (!b) return RMT_EINVAL;
  BCK(b, cudaStreamSynchronize(b->s));
  for (rmt_grid* m : b->g) {
    rmt_status st = grid_check(m);
    if (st != RMT_OK) return bfail(b, st, "member: %s", rmt_last_error(m));
  }
  return RMT_OK;
}

int rmt_batch_size(const rmt_batch* b) { return b ? (int)b->g.size() : 0; }

rmt_status rmt_batch_destroy(rmt_batch* b) {
  if (!b) return RMT_EINVAL;
  if (b->s) cudaStreamSynchronize(b->s);
  else cudaDeviceSynchronize();
  drop(b);
  for (size_t i = 0; i < b->g.size(); i++) {
    grid_leave_batch(b->g[i]);
    cudaStreamDestroy(b->bs[i]);
    cudaEventDestroy(b->join[i]);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
  return RMT_OK;
}

const char* rmt_batch_last_error(const rmt_batch* b) { return b ? b->msg : "null batch"; }

}  // extern "C"

// ============================================================================= serving

namespace {

struct Job {
  int id = 0;
  rmt_grid_desc desc;
  std::vector<rmt_solid_desc> solids;
  long steps_total = 0, steps_done = 0;
  size_t bytes = 0;
  int state = RMT_JOB_QUEUED;
  rmt_status status = RMT_OK;
  double t_submit = 0, t_admit = -1, t_done = -1;
  int last_slot = -1;  // event slot of the job's last launched step
  rmt_grid* g = nullptr;
  std::string msg;
};

constexpr int SLOTS = 2;  // steps in flight

}  // namespace

struct rmt_server {
  size_t budget = 0, used = 0;
  cudaStream_t s = nullptr;
  rmt_batch* batch = nullptr;
  std::map<int, Job*> jobs;
  std::deque<Job*> queue;
  std::vector<Job*> running;
  std::vector<std::pair<std::string, double>> options;
  cudaEvent_t ref = nullptr;     // GPU time origin (recorded and waited for at creation)
  cudaEvent_t ev[SLOTS] = {};    // end of the last steps (timing enabled)
  bool ev_used[SLOTS] = {};
  long nstep = 0;
  std::chrono::steady_clock::time_point t0;
  int next_id = 0;
  long steps_launched = 0;
  double cell_steps = 0;  // cells x steps of all launched job steps
  double admit_s = 0, retire_s = 0;  // host time spent admitting (create + initialise) and retiring
  char msg[512] = {0};
};

namespace {

double now(const rmt_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// seconds from the server's origin to the completion of the step recorded in slot k
double gpu_time(rmt_server* s, int k) {
  float ms = 0.f;
  if (cudaEventSynchronize(s->ev[k]) != cudaSuccess) return now(s);
  if (cudaEventElapsedTime(&ms, s->ref, s->ev[k]) != cudaSuccess) return now(s);
  return 1e-3 * ms;
}

void finish(rmt_server* s, Job* j, rmt_status st) {
  j->status = st;
  j->state = st == RMT_OK ? RMT_JOB_DONE : RMT_JOB_FAILED;
  if (j->g && st != RMT_OK) j->msg = rmt_last_error(j->g);
}

}  // namespace

extern "C" {

rmt_status rmt_server_create(size_t budget_bytes, void* stream, rmt_server** out) {
  if (!out || budget_bytes == 0) return RMT_EINVAL;
  *out = nullptr;
  rmt_server* s = new (std::nothrow) rmt_server();
  if (!s) return RMT_ENOMEM;
  s->budget = budget_bytes;
  s->s = (cudaStream_t)stream;
  s->t0 = std::chrono::steady_clock::now();
  rmt_status st = rmt_batch_create(stream, &s->batch);
  if (st == RMT_OK && cudaEventCreate(&s->ref) != cudaSuccess) st = RMT_ECUDA;
  for (int k = 0; k < SLOTS && st == RMT_OK; k++)
    if (cudaEventCreate(&s->ev[k]) != cudaSuccess) st = RMT_ECUDA;
  if (st == RMT_OK && (cudaEventRecord(s->ref, s->s) != cudaSuccess || cudaEventSynchronize(s->ref) != cudaSuccess))
    st = RMT_ECUDA;
  if (st != RMT_OK) {
    rmt_server_destroy(s);
    return st;
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return RMT_OK;
}

rmt_status rmt_server_set_option(rmt_server* s, const char* name, double value) {
  if (!s || !name) return RMT_EINVAL;
  s->options.push_back({name, value});
  return RMT_OK;
}

rmt_status rmt_server_submit(rmt_server* s, const rmt_grid_desc* d, const rmt_solid_desc* solids, int nsolids,
                             long nsteps, int* job_id) {
  if (!s || !d || nsteps < 0 || nsolids < 0 || (nsolids > 0 && !solids)) return RMT_EINVAL;
  if (d->mg_fixed_cycles <= 0 || d->mg_fixed_cycles_fe <= 0) return RMT_EINVAL;  // no host sync inside a step
  const size_t fp = rmt_grid_footprint(d, nsolids);
  if (fp == 0 || fp > s->budget) return RMT_EINVAL;
  Job* j = new (std::nothrow) Job();
  if (!j) return RMT_ENOMEM;
  j->id = s->next_id++;
  j->desc = *d;
  j->desc.cuda_stream = s->s;
  j->solids.assign(solids, solids + nsolids);
  j->steps_total = nsteps;
  j->bytes = fp;
  j->t_submit = now(s);
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  if (job_id) *job_id = j->id;
  return RMT_OK;
}

rmt_status rmt_server_poll(rmt_server* s, int* n_running, int* n_queued) {
  if (!s) return RMT_EINVAL;
  // 1. evict the jobs whose device error words report a failure (a diverged velocity, a
  //    degenerate extrapolation), freeing their memory, and retire the jobs whose last step has
  //    been launched; the others carry on
  const double t_ret = now(s);
  for (size_t i = 0; i < s->running.size();) {
    Job* j = s->running[i];
    const rmt_status fs = grid_poll(j->g);
    if (fs != RMT_OK) {
      rmt_batch_remove(s->batch, j->g);
      finish(s, j, fs);
      j->t_done = now(s);
      rmt_destroy_grid(j->g);
      j->g = nullptr;
      s->used -= j->bytes;
      s->running.erase(s->running.begin() + i);
      continue;
    }
    if (j->steps_done < j->steps_total) {
      i++;
      continue;
    }
    j->t_done = j->last_slot >= 0 ? gpu_time(s, j->last_slot) : now(s);
    if (rmt_batch_size(s->batch) > 0) rmt_batch_remove(s->batch, j->g);  // not a member any more: no-op
    finish(s, j, grid_check(j->g));
    s->running.erase(s->running.begin() + i);
  }
  s->retire_s += now(s) - t_ret;
  // 2. admit queued jobs in arrival order while they fit (a job that does not fit waits; later
  //    smaller ones may pass it)
  const double t_adm = now(s);
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Job* j = *it;
    if (s->used + j->bytes > s->budget) {
      ++it;
      continue;
    }
    it = s->queue.erase(it);
    j->t_admit = now(s);
    rmt_status st = rmt_create_grid(&j->desc, &j->g);
    for (size_t q = 0; q < j->solids.size() && st == RMT_OK; q++) st = rmt_add_solid(j->g, &j->solids[q], nullptr);
    for (const auto& o : s->options)
      if (st == RMT_OK) st = rmt_set_option(j->g, o.first.c_str(), o.second);
    if (st == RMT_OK) st = rmt_batch_add(s->batch, j->g);
    if (st != RMT_OK) {
      // the job fails alone; the others carry on
      j->msg = j->g ? rmt_last_error(j->g) : "invalid grid description";
      if (j->g) {
        rmt_destroy_grid(j->g);
        j->g = nullptr;
      }
      j->status = st;
      j->state = RMT_JOB_FAILED;
      j->t_done = now(s);
      continue;
    }
    s->used += j->bytes;
    j->state = RMT_JOB_RUNNING;
    s->running.push_back(j);
  }
  s->admit_s += now(s) - t_adm;
  // 3. one batched step of the running jobs (at most SLOTS steps in flight)
  std::vector<Job*> stepping;
  for (Job* j : s->running)
    if (j->steps_done < j->steps_total) stepping.push_back(j);
  if (!stepping.empty()) {
    const int k = (int)(s->nstep % SLOTS);
    if (s->ev_used[k]) cudaEventSynchronize(s->ev[k]);
    // a job admitted with zero steps is the only member that is not stepping: it leaves first
    for (Job* j : s->running)
      if (j->steps_done >= j->steps_total) rmt_batch_remove(s->batch, j->g);
    rmt_status st = rmt_batch_step(s->batch, 1);
    if (st != RMT_OK) {
      snprintf(s->msg, sizeof s->msg, "batched step: %s", rmt_batch_last_error(s->batch));
      return st;
    }
    const cudaError_t e = cudaEventRecord(s->ev[k], s->s);
    if (e != cudaSuccess) {
      snprintf(s->msg, sizeof s->msg, "event record: %s", cudaGetErrorString(e));
      return RMT_ECUDA;
    }
    s->ev_used[k] = true;
    s->nstep++;
    s->steps_launched++;
    for (Job* j : stepping) {
      j->steps_done++;
      j->last_slot = k;
      s->cell_steps += (double)j->desc.n[0] * j->desc.n[1] * j->desc.n[2];
    }
  }
  if (n_running) *n_running = (int)s->running.size();
  if (n_queued) *n_queued = (int)s->queue.size();
  return RMT_OK;
}

rmt_status rmt_server_job(rmt_server* s, int id, rmt_job_info* info) {
  if (!s || !info) return RMT_EINVAL;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RMT_EINVAL;
  const Job* j = it->second;
  info->state = j->state;
  info->status = j->status;
  info->steps_done = j->steps_done;
  info->steps_total = j->steps_total;
  info->t_submit = j->t_submit;
  info->t_admit = j->t_admit;
  info->t_done = j->t_done;
  info->device_bytes = j->bytes;
  return RMT_OK;
}

rmt_grid* rmt_server_job_grid(rmt_server* s, int id) {
  if (!s) return nullptr;
  auto it = s->jobs.find(id);
  return it == s->jobs.end() ? nullptr : it->second->g;
}

rmt_status rmt_server_release(rmt_server* s, int id) {
  if (!s) return RMT_EINVAL;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RMT_EINVAL;
  Job* j = it->second;
  if (j->state == RMT_JOB_RUNNING || j->state == RMT_JOB_QUEUED) return RMT_ESTATE;
  if (j->g) {
    rmt_destroy_grid(j->g);
    j->g = nullptr;
    s->used -= j->bytes;
  }
  delete j;
  s->jobs.erase(it);
  return RMT_OK;
}

size_t rmt_server_resident_bytes(const rmt_server* s) { return s ? s->used : 0; }
const char* rmt_server_last_error(const rmt_server* s) { return s ? s->msg : "null server"; }

rmt_status rmt_server_stats(const rmt_server* s, rmt_server_stats_t* out) {
  if (!s || !out) return RMT_EINVAL;
  out->batched_steps = s->steps_launched;
  out->graph_captures = s->batch ? s->batch->captures : 0;
  out->capture_s = s->batch ? s->batch->capture_s : 0.0;
  out->admit_s = s->admit_s;
  out->retire_s = s->retire_s;
  out->cell_steps = s->cell_steps;
  return RMT_OK;
}
double rmt_server_clock(const rmt_server* s) { return s ? now(s) : 0.0; }
double rmt_server_cell_steps(const rmt_server* s) { return s ? s->cell_steps : 0.0; }

rmt_status rmt_server_destroy(rmt_server* s) {
  if (!s) return RMT_EINVAL;
  if (s->s) cudaStreamSynchronize(s->s);
  if (s->batch) rmt_batch_destroy(s->batch);
  for (auto& kv : s->jobs) {
    if (kv.second->g) rmt_destroy_grid(kv.second->g);
    delete kv.second;
  }
  if (s->ref) cudaEventDestroy(s->ref);
  for (int k = 0; k < SLOTS; k++)
    if (s->ev[k]) cudaEventDestroy(s->ev[k]);
  delete s;
  return RMT_OK;
}

}  // extern "C"
