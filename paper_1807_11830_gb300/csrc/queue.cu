// Serving: a request queue with continuous (iteration-level) batching.
//
// Submitted reconstructions wait in arrival order.  A scheduler thread
// admits them while the device-memory budget and the live-request limit
// allow (strict arrival order: the head of the queue blocks those behind
// it), uploads their inputs, starts CG (b = E^H y) and then ticks: each tick
// advances every live frame by one CG iteration, with one persistent launch
// per size class whose frame table holds the live frames of every request of
// that class, each at its own iteration.  After a tick the scheduler reads
// back which frames are still iterating; requests whose frames have all
// stopped, or that reached max_iter, or were cancelled, retire: their image
// is copied to pinned host memory and their device memory is freed, making
// room for the next admissions.
//
// fake_device mode runs the same scheduler with no GPU work (each tick
// sleeps; every frame stops after min(max_iter, fake_iters) ticks), so
// admission, ordering, refusal and cancellation are testable on a CPU.
//
// With SENSE_QUEUE_LOG set to a path, every request that leaves the queue
// appends one JSON line there: its shape, final state and status, the times
// of submission, admission, end of its first tick and completion (ms since
// the queue was created), ticks applied, largest per-frame iteration count
// and relative residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "launch.h"
#include "pinned.h"
#include "plan.h"
#include "trace.h"
#include "sense.h"
#include "sense_testing.h"

using namespace sense;
using Clock = std::chrono::steady_clock;

namespace {

__global__ void k_gather_active(const PFrame* table, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __ldcg(table[i].active);
}

struct Request {
  uint64_t id = 0;
  sense_shape sh{};
  int max_iter = 0;
  double tol = 0.0;
  size_t need = 0;      // device bytes reserved for it
  size_t y_bytes = 0, s_bytes = 0, l_bytes = 0, x_bytes = 0;
  // pinned host staging (inputs at submit, outputs at retirement)
  void* y_h = nullptr;
  void* s_h = nullptr;
  int* lines_h = nullptr;
  float2* x_h = nullptr;
  int* iters_h = nullptr;
  double* resid_h = nullptr;
  int* outcome_h = nullptr;
  // device
  sense_plan* plan = nullptr;
  void* y_d = nullptr;
  void* s_d = nullptr;
  const void* maps = nullptr;  // what its normal-operator tiles read: s_d or the plan's S^T
  int* lines_d = nullptr;
  float2* x_d = nullptr;
  int* out_i_d = nullptr;  // iters [F], outcome [F]
  double* resid_d = nullptr;
  int* err_h = nullptr;     // device error flags of its plan, read at retirement
  int ticks = 0;            // CG iterations applied (capped at max_iter)
  int state = SENSE_REQ_PENDING;
  bool cancel = false;
  int status_off = 0;  // position of its frames in the tick's status array
  double waves = -1.0;  // normal-operator work per CG iteration in waves of resident blocks (at admission)
  int cls = -1;
  Clock::time_point t_submit, t_admit, t_first, t_done;
  bool admitted = false, ticked = false;
  sense_status fail_status = SENSE_ECUDA;  // what sense_queue_wait reports for a failed request
  std::string fail_msg = "request failed on the device";
};

struct SizeClass {
  int ny = 0, nx = 0, storage = 0, variant = -1;
  int cap = 0;  // frames the buffers hold
  int* ints = nullptr;
  double* part_nrm = nullptr;
  double* part_upd = nullptr;
  int upd_cap = 0;  // chunks per frame the buffer holds
  PFrame* table_d = nullptr;
  PFrame* table_h = nullptr;  // pinned
  int* status_d = nullptr;
  int* status_h = nullptr;  // pinned
  cudaStream_t stream = nullptr;  // its persistent launches overlap those of other classes
  cudaEvent_t done = nullptr;
};

size_t elem_bytes(int storage) { return storage == SENSE_STORE_BF16 ? 4 : 8; }

}  // namespace

struct sense_queue {
  int device = 0;
  sense_queue_cfg cfg{};
  sense_queue_test_hooks hooks{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> live;  // worker thread only
  std::map<uint64_t, Request*> reqs;
  uint64_t next_id = 1;
  size_t budget = 0, in_use = 0;
  bool stop = false;
  std::thread worker;
  sense_queue_stats st{};
  std::vector<double> lat_ms;
  uint64_t admissions = 0;      // counts admissions for the fail_admit_every test hook
  double iter_ms = 0.0;         // last tick's time per CG iteration (worker thread)
  double gap_ms = 0.0;          // running mean of the time between submissions (under mu)
  Clock::time_point last_submit;
  bool any_submit = false;
  cudaEvent_t admitted = nullptr;  // recorded after each round of admissions
  FILE* log = nullptr;          // per-request JSON lines (SENSE_QUEUE_LOG), written under mu
  Clock::time_point t0;         // creation time, origin of the logged times
  cudaStream_t stream = nullptr;
  int sms = 0;
  std::map<std::tuple<int, int, int>, SizeClass> classes;  // worker thread only
  std::map<std::tuple<int, int, int>, int> variants;         // guarded by mu
  std::map<int, float2*> twiddles;                            // device tables per length (worker thread)
  // host staging of inputs and outputs (page-locked unless fake_device)
  std::unique_ptr<PinnedArena> arena;
};

namespace {

// Input staging is released once the request's uploads have completed.
void free_host(sense_queue* q, Request* r) {
  q->arena->put(r->y_h);
  q->arena->put(r->s_h);
  q->arena->put(r->lines_h);
  r->y_h = r->s_h = nullptr;
  r->lines_h = nullptr;
}

void free_outputs(sense_queue* q, Request* r) {
  q->arena->put(r->x_h);
  q->arena->put(r->iters_h);
  q->arena->put(r->resid_h);
  q->arena->put(r->outcome_h);
  q->arena->put(r->err_h);
  r->err_h = nullptr;
  r->x_h = nullptr;
  r->iters_h = nullptr;
  r->resid_h = nullptr;
  r->outcome_h = nullptr;
}

// Stream-ordered release of a request's device memory (no device-wide sync).
void free_device(Request* r, cudaStream_t st) {
  if (r->plan) plan_destroy_pooled(r->plan);
  r->plan = nullptr;
  for (void* p : {r->y_d, r->s_d, (void*)r->lines_d, (void*)r->x_d, (void*)r->out_i_d, (void*)r->resid_d})
    if (p) cudaFreeAsync(p, st);
  r->y_d = r->s_d = nullptr;
  r->lines_d = nullptr;
  r->x_d = nullptr;
  r->out_i_d = nullptr;
  r->resid_d = nullptr;
}

// Device bytes a request holds while live: its inputs, output and the plan's
// workspace (CG vectors, the k-space intermediate, scalars, the transposed
// maps that lane-major kernel variants read), with slack.
size_t request_need(const sense_shape& sh) {
  const size_t F = sh.frames, img = (size_t)sh.ny * sh.nx;
  const size_t e = elem_bytes(sh.storage);
  const size_t inputs = F * sh.coils * sh.lines * sh.nx * e + (size_t)sh.coils * img * e + F * sh.lines * 4;
  const size_t outputs = F * img * 8 + F * 16;
  const size_t plan = F * sh.coils * sh.lines * sh.nx * 8 + 4 * F * img * 8 + (size_t)sh.coils * img * e;
  return inputs + outputs + plan + (size_t)(1 << 20);
}

double ms_since(const sense_queue* q, Clock::time_point t) {
  return std::chrono::duration<double, std::milli>(t - q->t0).count();
}

// One JSON line per request leaving the queue (caller holds q->mu).
void log_request(sense_queue* q, const Request* r) {
  if (!q->log) return;
  static const char* kState[] = {"pending", "running", "done", "cancelled", "failed"};
  const int s = (r->state >= 0 && r->state <= SENSE_REQ_FAILED) ? r->state : SENSE_REQ_FAILED;
  const int status = r->state == SENSE_REQ_FAILED ? (int)r->fail_status : 0;
  std::fprintf(q->log,
               "{\"id\": %llu, \"ny\": %d, \"nx\": %d, \"coils\": %d, \"frames\": %d, \"lines\": %d, "
               "\"storage\": \"%s\", \"centred\": %d, \"state\": \"%s\", \"status\": %d, \"submit_ms\": %.3f",
               (unsigned long long)r->id, r->sh.ny, r->sh.nx, r->sh.coils, r->sh.frames, r->sh.lines,
               r->sh.storage == SENSE_STORE_BF16 ? "bf16" : "c64", r->sh.centred, kState[s], status,
               ms_since(q, r->t_submit));
  if (r->admitted) std::fprintf(q->log, ", \"admit_ms\": %.3f", ms_since(q, r->t_admit));
  if (r->ticked) std::fprintf(q->log, ", \"first_tick_ms\": %.3f", ms_since(q, r->t_first));
  std::fprintf(q->log, ", \"done_ms\": %.3f, \"latency_ms\": %.3f, \"ticks\": %d, \"max_iter\": %d",
               ms_since(q, r->t_done), std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count(),
               r->ticks, r->max_iter);
  if (r->state == SENSE_REQ_DONE && r->iters_h && r->resid_h) {
    int it = 0;
    double res = 0.0;
    bool finite = true;
    for (int f = 0; f < r->sh.frames; ++f) {
      it = std::max(it, r->iters_h[f]);
      if (std::isfinite(r->resid_h[f]))
        res = std::max(res, r->resid_h[f]);
      else
        finite = false;
    }
    if (finite)
      std::fprintf(q->log, ", \"iters\": %d, \"max_rel_resid\": %.6e", it, res);
    else
      std::fprintf(q->log, ", \"iters\": %d, \"max_rel_resid\": null", it);
  }
  std::fputs("}\n", q->log);
  std::fflush(q->log);
}

// Work of a request per CG iteration, in coil-pixels: frames x coils x ny x nx.
double request_work(const sense_shape& sh) { return (double)sh.frames * sh.coils * sh.ny * sh.nx; }

// Normal-operator work of a request per CG iteration in waves of the device:
// frames x column tiles of its size class's kernel variant, over the blocks
// that variant's persistent kernel keeps resident (SMs x blocks per SM).
// Called by the worker thread with q->mu held (reads the class variants).
double request_waves(sense_queue* q, const sense_shape& sh) {
  static std::map<std::tuple<int, int, int>, int> resident;  // (ny, variant, storage) -> blocks per SM
  int variant = 0;
  auto it = q->variants.find(std::make_tuple(sh.ny, sh.nx, sh.storage));
  if (it != q->variants.end() && it->second >= 0) variant = it->second;
  int W = normal_variant_width(sh.ny, variant);
  if (W <= 0) W = 8;
  int per_sm = 2;
  if (!q->hooks.fake_device) {
    const auto key = std::make_tuple(sh.ny, variant, sh.storage);
    auto rt = resident.find(key);
    if (rt == resident.end()) {
      int occ = cg_persistent_resident(sh.ny, variant, sh.storage == SENSE_STORE_BF16);
      rt = resident.emplace(key, occ > 0 ? occ : 1).first;
    }
    per_sm = rt->second;
  }
  const int sms = q->sms > 0 ? q->sms : 152;
  const double tiles = (double)((sh.nx + W - 1) / W);
  return (double)sh.frames * tiles / ((double)sms * per_sm);
}

void record_done(sense_queue* q, Request* r, int state) {
  std::lock_guard<std::mutex> lock(q->mu);
  r->state = state;
  r->t_done = Clock::now();
  log_request(q, r);
  if (state == SENSE_REQ_DONE) {
    q->st.completed++;
    q->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  } else if (state == SENSE_REQ_CANCELLED) {
    q->st.cancelled++;
  } else {
    q->st.failed++;
  }
  q->in_use -= std::min(q->in_use, r->need);
  q->cv_done.notify_all();
  q->cv_work.notify_all();
}

bool ensure_class_capacity(sense_queue* q, SizeClass& c, int frames) {
  if (!c.stream && (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess))
    return false;
  if (c.cap >= frames && c.upd_cap > 0) return true;
  int cap = std::max(frames, std::max(64, c.cap * 2));
  // free the old buffers (the stream is idle between ticks)
  for (void* p : {(void*)c.ints, (void*)c.part_nrm, (void*)c.part_upd, (void*)c.table_d, (void*)c.status_d})
    if (p) cudaFree(p);
  if (c.table_h) cudaFreeHost(c.table_h);
  if (c.status_h) cudaFreeHost(c.status_h);
  int min_threads = 1 << 30;
  for (int v = 0; v < kNormVariants; ++v) {
    const int th = normal_variant_threads(c.ny, v);
    if (th > 0) min_threads = std::min(min_threads, th);
  }
  c.upd_cap = update_chunks((size_t)c.ny * c.nx, min_threads);
  bool ok = cudaMalloc(&c.ints, sizeof(int) * (4 * (size_t)cap + 1)) == cudaSuccess &&
            cudaMalloc(&c.part_nrm, sizeof(double) * (size_t)cap * ((c.nx + 3) / 4)) == cudaSuccess &&
            cudaMalloc(&c.part_upd, sizeof(double) * (size_t)cap * c.upd_cap) == cudaSuccess &&
            cudaMalloc(&c.table_d, sizeof(PFrame) * cap) == cudaSuccess &&
            cudaMalloc(&c.status_d, sizeof(int) * cap) == cudaSuccess &&
            cudaMallocHost(&c.table_h, sizeof(PFrame) * cap) == cudaSuccess &&
            cudaMallocHost(&c.status_h, sizeof(int) * cap) == cudaSuccess;
  c.cap = ok ? cap : 0;
  return ok;
}

const float2* twiddle_table(sense_queue* q, int n) {
  auto it = q->twiddles.find(n);
  if (it != q->twiddles.end()) return it->second;
  const std::vector<float2> host = plan_twiddles(n);
  float2* d = nullptr;
  if (cudaMalloc(&d, sizeof(float2) * n) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, host.data(), sizeof(float2) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  q->twiddles[n] = d;
  return d;
}

// Upload inputs, create the plan (stream-ordered workspace, shared twiddle
// tables), start CG.  Everything is queued on the queue's stream; nothing
// synchronises.  Returns false on failure.
// inject_fail (test hook): fail as if the last device allocation had failed,
// after the others succeeded, so the partial clean-up runs.
bool admit_device(sense_queue* q, Request* r, std::string* err, bool inject_fail) {
  sense::TraceRange trace_range("sense_queue_admit");
  const sense_shape& sh = r->sh;
  const size_t F = sh.frames;
  cudaStream_t st = q->stream;
  const float2* twy = twiddle_table(q, sh.ny);
  const float2* twx = twiddle_table(q, sh.nx);
  if (!twy || !twx) {
    *err = "twiddle table set-up failed";
    return false;
  }
  if (plan_create_pooled(&sh, q->device, st, twy, twx, &r->plan) != SENSE_OK) {
    *err = sense_last_error();
    return false;
  }
  r->plan->cg_mode = 1;
  bool ok = cudaMallocAsync(&r->y_d, r->y_bytes, st) == cudaSuccess &&
            cudaMallocAsync(&r->s_d, r->s_bytes, st) == cudaSuccess &&
            cudaMallocAsync((void**)&r->lines_d, r->l_bytes, st) == cudaSuccess &&
            cudaMallocAsync((void**)&r->x_d, r->x_bytes, st) == cudaSuccess &&
            cudaMallocAsync((void**)&r->out_i_d, sizeof(int) * 2 * F, st) == cudaSuccess &&
            cudaMallocAsync((void**)&r->resid_d, sizeof(double) * F, st) == cudaSuccess;
  if (ok && inject_fail) {
    *err = "device allocation failed (injected by the fail_admit_every test hook)";
    return false;
  }
  if (!ok) {
    cudaGetLastError();
    *err = "device allocation failed";
    return false;
  }
  ok = cudaMemcpyAsync(r->y_d, r->y_h, r->y_bytes, cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(r->s_d, r->s_h, r->s_bytes, cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(r->lines_d, r->lines_h, r->l_bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) {
    *err = "input upload failed";
    return false;
  }
  // kernel variant of the size class: autotuned on its first request, then fixed
  const auto key = std::make_tuple(sh.ny, sh.nx, sh.storage);
  int variant = -1;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    auto it = q->variants.find(key);
    if (it != q->variants.end()) variant = it->second;
  }
  if (variant < 0) {
    variant = 0;
    if (q->cfg.autotune) {
      int v = 0;
      if (sense_plan_autotune(r->plan, r->s_d, r->lines_d, &v, nullptr, st) == SENSE_OK) variant = v;
    }
    std::lock_guard<std::mutex> lock(q->mu);
    q->variants[key] = variant;
  }
  if (plan_set_variant_nosync(r->plan, variant) != SENSE_OK) {
    *err = sense_last_error();
    return false;
  }
  if (!plan_maps_transposed(r->plan) && plan_prepare_tmap(r->plan, r->s_d, st) != SENSE_OK) {
    *err = sense_last_error();
    return false;
  }
  if (plan_maps(r->plan, r->s_d, st, &r->maps) != SENSE_OK) {
    *err = sense_last_error();
    return false;
  }
  if (plan_cg_start(r->plan, r->y_d, r->s_d, r->lines_d, r->x_d, r->tol, st) != SENSE_OK) {
    *err = sense_last_error();
    return false;
  }
  return true;
}

// Queue the result copies of a finished request (to its pinned buffers).
bool retire_enqueue(sense_queue* q, Request* r) {
  const size_t F = r->sh.frames;
  cudaStream_t st = q->stream;
  bool ok = plan_cg_finish(r->plan, r->out_i_d, r->resid_d, r->out_i_d + F, st) == SENSE_OK;
  ok = ok && plan_centred_output(r->plan, r->x_d, st) == SENSE_OK;
  ok = ok && cudaMemcpyAsync(r->x_h, r->x_d, r->x_bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(r->iters_h, r->out_i_d, sizeof(int) * F, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(r->outcome_h, r->out_i_d + F, sizeof(int) * F, cudaMemcpyDeviceToHost, st) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(r->resid_h, r->resid_d, sizeof(double) * F, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(r->err_h, r->plan->err(), sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  return ok;
}

// One tick: iters_per_tick CG iterations of every live frame, one persistent
// launch per size class; frames stop at their own max_iter / tolerance inside
// the launch.  Then one stream synchronisation reads back which frames still
// iterate; finished requests queue their result copies, a second
// synchronisation completes those, and their memory is released in stream
// order.
bool tick_device(sense_queue* q) {
  sense::TraceRange trace_range("sense_queue_tick");
  // Iterations per tick: the configured number, or by default
  //  * while requests wait for admission, what fits in kWaitTickMs at the
  //    last tick's time per iteration (1 to 10), so they join soon;
  //  * otherwise 10, stretched up to the largest remaining budget of the live
  //    requests (at most 80) so a lone request is not cut into many host
  //    round trips, but no longer than the recent mean time between
  //    submissions (at least kWaitTickMs): the next arrival is then likely
  //    to come during the tick and should not wait long for its end.
  constexpr double kWaitTickMs = 4.0;
  int m = q->cfg.iters_per_tick > 0 ? q->cfg.iters_per_tick : 10;
  if (q->cfg.iters_per_tick <= 0) {
    bool waiting;
    double gap;
    {
      std::lock_guard<std::mutex> lock(q->mu);
      waiting = !q->pending.empty();
      gap = q->gap_ms;
    }
    if (!waiting) {
      int remaining = 0;
      for (Request* r : q->live) remaining = std::max(remaining, r->max_iter - r->ticks);
      m = std::max(m, std::min(remaining, 8 * m));
      if (q->iter_ms > 0.0 && gap > 0.0)
        m = (int)std::max(1.0, std::min((double)m, std::floor(std::max(kWaitTickMs, gap) / q->iter_ms)));
    } else if (q->iter_ms > 0.0) {
      m = (int)std::max(1.0, std::min((double)m, std::floor(kWaitTickMs / q->iter_ms)));
    }
  }
  const Clock::time_point t_tick = Clock::now();
  // the admissions just queued on q->stream come before every class's launch
  if (cudaEventRecord(q->admitted, q->stream) != cudaSuccess) return false;
  std::map<std::tuple<int, int, int>, std::vector<Request*>> by_class;
  for (Request* r : q->live) by_class[std::make_tuple(r->sh.ny, r->sh.nx, r->sh.storage)].push_back(r);
  std::vector<std::pair<SizeClass*, int>> launched;
  for (auto& kv : by_class) {
    SizeClass& c = q->classes[kv.first];
    c.ny = std::get<0>(kv.first);
    c.nx = std::get<1>(kv.first);
    c.storage = std::get<2>(kv.first);
    int frames = 0;
    for (Request* r : kv.second) frames += r->sh.frames;
    if (!ensure_class_capacity(q, c, frames)) return false;
    int off = 0;
    for (Request* r : kv.second) {
      r->status_off = off;
      plan_frames(r->plan, r->maps, r->lines_d, r->x_d, r->ticks, r->tol, c.table_h + off, off);
      for (int f = 0; f < r->sh.frames; ++f) c.table_h[off + f].kmax = r->max_iter;
      off += r->sh.frames;
    }
    const int variant = sense_plan_variant(kv.second[0]->plan);
    const int W = normal_variant_width(c.ny, variant);
    const int th = normal_variant_threads(c.ny, variant);
    PArgs a{};
    a.frames = c.table_d;
    a.nframes = frames;
    a.nx = c.nx;
    a.tiles = (c.nx + W - 1) / W;
    a.chunks = update_chunks((size_t)c.ny * c.nx, th);
    a.lag = persistent_order(c.table_h, frames);
    a.iters = m;
    a.ticket = reinterpret_cast<unsigned*>(c.ints + 4 * frames);
    a.tw = kv.second[0]->plan->tw_y;
    a.err = kv.second[0]->plan->err();
    a.st.nrm_arrive = reinterpret_cast<unsigned*>(c.ints);
    a.st.upd_arrive = reinterpret_cast<unsigned*>(c.ints + frames);
    a.st.nrm_ready = c.ints + 2 * frames;
    a.st.upd_ready = c.ints + 3 * frames;
    a.st.part_nrm = c.part_nrm;
    a.st.part_upd = c.part_upd;
    if (a.chunks > c.upd_cap) return false;
    // each class on its own stream: the launches of different classes overlap
    // (each kernel's blocks wait only on blocks of the same launch)
    cudaStream_t cs = c.stream;
    bool ok = cudaStreamWaitEvent(cs, q->admitted, 0) == cudaSuccess &&
              cudaMemcpyAsync(c.table_d, c.table_h, sizeof(PFrame) * frames, cudaMemcpyHostToDevice, cs) ==
                  cudaSuccess &&
              cudaMemsetAsync(c.ints, 0, sizeof(int) * (4 * (size_t)frames + 1), cs) == cudaSuccess;
    cudaError_t e = c.storage == SENSE_STORE_BF16 ? launch_cg_persistent<StBF16>(c.ny, variant, a, q->sms, cs)
                                                  : launch_cg_persistent<StC64>(c.ny, variant, a, q->sms, cs);
    if (!ok || e != cudaSuccess) return false;
    k_gather_active<<<(frames + 255) / 256, 256, 0, cs>>>(c.table_d, frames, c.status_d);
    if (cudaMemcpyAsync(c.status_h, c.status_d, sizeof(int) * frames, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaEventRecord(c.done, cs) != cudaSuccess || cudaStreamWaitEvent(q->stream, c.done, 0) != cudaSuccess)
      return false;
    for (Request* r : kv.second) r->cls = (int)launched.size();
    launched.emplace_back(&c, frames);
  }
  if (cudaStreamSynchronize(q->stream) != cudaSuccess) return false;
  q->iter_ms = std::chrono::duration<double, std::milli>(Clock::now() - t_tick).count() / m;
  for (Request* r : q->live)
    if (r->y_h) free_host(q, r);  // its uploads, queued before this tick, have completed
  std::vector<Request*> still, finished, cancelled;
  const Clock::time_point now = Clock::now();
  for (Request* r : q->live) {
    r->ticks = std::min(r->ticks + m, r->max_iter);
    if (!r->ticked) {
      r->ticked = true;
      r->t_first = now;
    }
    const SizeClass* c = launched[r->cls].first;
    bool any = false;
    for (int f = 0; f < r->sh.frames; ++f) any |= c->status_h[r->status_off + f] != 0;
    bool cancel;
    {
      std::lock_guard<std::mutex> lock(q->mu);
      cancel = r->cancel;
    }
    if (cancel)
      cancelled.push_back(r);
    else if (!any || r->ticks >= r->max_iter)
      finished.push_back(r);
    else
      still.push_back(r);
  }
  std::vector<bool> ok(finished.size());
  for (size_t i = 0; i < finished.size(); ++i) ok[i] = retire_enqueue(q, finished[i]);
  if (!finished.empty() && cudaStreamSynchronize(q->stream) != cudaSuccess)
    for (size_t i = 0; i < finished.size(); ++i) ok[i] = false;
  for (size_t i = 0; i < finished.size(); ++i) {
    Request* r = finished[i];
    free_device(r, q->stream);
    record_done(q, r, (ok[i] && *r->err_h == 0) ? SENSE_REQ_DONE : SENSE_REQ_FAILED);
  }
  for (Request* r : cancelled) {
    free_device(r, q->stream);
    record_done(q, r, SENSE_REQ_CANCELLED);
  }
  q->live.swap(still);
  return true;
}

void tick_fake(sense_queue* q) {
  if (q->hooks.fake_tick_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(q->hooks.fake_tick_us));
  std::vector<Request*> still;
  const Clock::time_point now = Clock::now();
  for (Request* r : q->live) {
    r->ticks++;
    if (!r->ticked) {
      r->ticked = true;
      r->t_first = now;
    }
    bool cancel;
    {
      std::lock_guard<std::mutex> lock(q->mu);
      cancel = r->cancel;
    }
    const int stop_at = std::min(r->max_iter, q->hooks.fake_iters > 0 ? q->hooks.fake_iters : r->max_iter);
    if (cancel) {
      record_done(q, r, SENSE_REQ_CANCELLED);
    } else if (r->ticks >= stop_at) {
      const size_t F = r->sh.frames;
      memset(r->x_h, 0, r->x_bytes);
      for (size_t f = 0; f < F; ++f) {
        r->iters_h[f] = r->ticks;
        r->outcome_h[f] = r->ticks >= r->max_iter ? SENSE_CG_MAXITER : SENSE_CG_CONVERGED;
        r->resid_h[f] = 0.0;
      }
      free_host(q, r);
      record_done(q, r, SENSE_REQ_DONE);
    } else {
      still.push_back(r);
    }
  }
  q->live.swap(still);
}

constexpr double kDefaultAdmitWaves = 12.0;

void worker_main(sense_queue* q) {
  if (!q->hooks.fake_device) cudaSetDevice(q->device);
  for (;;) {
    std::vector<Request*> admit;
    const double work_cap = q->cfg.max_live_work > 0 ? (double)q->cfg.max_live_work : 1e300;
    const double waves_cap =
        q->cfg.admit_waves < 0.0 ? 1e300 : (q->cfg.admit_waves == 0.0 ? kDefaultAdmitWaves : q->cfg.admit_waves);
    double live_work = 0.0, live_waves = 0.0;
    for (const Request* r : q->live) {
      live_work += request_work(r->sh);
      live_waves += r->waves;
    }
    {
      std::unique_lock<std::mutex> lock(q->mu);
      q->cv_work.wait(lock, [&] { return q->stop || !q->pending.empty() || !q->live.empty(); });
      if (q->stop) break;
      while (!q->pending.empty()) {
        Request* r = q->pending.front();
        if (r->cancel) {
          q->pending.pop_front();
          r->state = SENSE_REQ_CANCELLED;
          r->t_done = Clock::now();
          q->st.cancelled++;
          log_request(q, r);
          q->cv_done.notify_all();
          continue;
        }
        const size_t n_live = q->live.size() + admit.size();
        if (q->cfg.max_live > 0 && (int)n_live >= q->cfg.max_live) break;
        if (q->in_use + r->need > q->budget) break;  // arrival order: the head waits for room
        // enough work live to fill the GPU: later requests wait, in arrival order, rather
        // than share every tick and all finish late (a lone request over the cap is admitted)
        if (live_work > 0 && live_work + request_work(r->sh) > work_cap) break;
        // saturation: enough normal-operator work is live to fill the device; the
        // head waits (arrival order) so the oldest requests finish first
        if (live_waves >= waves_cap) break;
        if (r->waves < 0.0) r->waves = request_waves(q, r->sh);
        live_waves += r->waves;
        live_work += request_work(r->sh);
        q->pending.pop_front();
        q->in_use += r->need;
        r->state = SENSE_REQ_RUNNING;
        r->admitted = true;
        r->t_admit = Clock::now();
        q->st.admitted++;
        admit.push_back(r);
      }
    }
    for (Request* r : admit) {
      std::string err;
      const bool inject = q->hooks.fail_admit_every > 0 && ++q->admissions % (uint64_t)q->hooks.fail_admit_every == 0;
      bool ok;
      if (q->hooks.fake_device) {
        ok = !inject;
        if (inject) err = "device allocation failed (injected by the fail_admit_every test hook)";
      } else {
        ok = admit_device(q, r, &err, inject);
      }
      if (ok) {
        q->live.push_back(r);
      } else {
        if (!q->hooks.fake_device) free_device(r, q->stream);
        r->fail_status = err.rfind("device allocation failed", 0) == 0 ? SENSE_ENOMEM : SENSE_ECUDA;
        r->fail_msg = "admission failed: " + err;
        record_done(q, r, SENSE_REQ_FAILED);
      }
    }
    if (q->live.empty()) continue;
    if (q->hooks.fake_device) {
      tick_fake(q);
    } else if (!tick_device(q)) {
      // launches already issued on the class streams may still read the requests' memory
      for (auto& kv : q->classes)
        if (kv.second.stream) cudaStreamSynchronize(kv.second.stream);
      for (Request* r : q->live) {
        free_device(r, q->stream);
        record_done(q, r, SENSE_REQ_FAILED);
      }
      q->live.clear();
    }
    std::lock_guard<std::mutex> lock(q->mu);
    q->st.ticks++;
  }
  // shutdown: cancel what is left
  for (Request* r : q->live) {
    if (!q->hooks.fake_device) free_device(r, q->stream);
    record_done(q, r, SENSE_REQ_CANCELLED);
  }
  q->live.clear();
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

sense_status qfail(sense_status s, const std::string& m) {
  record_error(m);
  return s;
}

}  // namespace

extern "C" {

sense_status sense_queue_create(int device, const sense_queue_cfg* cfg, sense_queue** out) {
  return sense_queue_create_with_hooks(device, cfg, nullptr, out);
}

sense_status sense_queue_create_with_hooks(int device, const sense_queue_cfg* cfg, const sense_queue_test_hooks* hooks,
                                           sense_queue** out) {
  if (!out) return qfail(SENSE_EINVAL, "out is NULL");
  *out = nullptr;
  if (hooks && hooks->fail_admit_every < 0) return qfail(SENSE_EINVAL, "fail_admit_every must be >= 0");
  if (cfg && !(cfg->admit_waves == cfg->admit_waves)) return qfail(SENSE_EINVAL, "admit_waves is NaN");
  sense_queue* q = new sense_queue();
  if (cfg) q->cfg = *cfg;
  if (hooks) q->hooks = *hooks;
  q->device = device;
  q->t0 = Clock::now();
  q->arena.reset(new PinnedArena(!q->hooks.fake_device));
  if (!q->arena->reserve(q->cfg.staging_reserve_bytes)) {
    delete q;
    return qfail(SENSE_ENOMEM, "staging reservation of page-locked host memory failed");
  }
  if (!q->hooks.fake_device) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
      delete q;
      return qfail(SENSE_EINVAL, "device index out of range (or no CUDA device)");
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    cudaDeviceGetAttribute(&q->sms, cudaDevAttrMultiProcessorCount, device);
    // keep freed request memory in the device's stream-ordered pool for reuse
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->admitted, cudaEventDisableTiming);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
      delete q;
      return qfail(SENSE_ECUDA, "queue stream creation failed");
    }
    const size_t reserve = (size_t)1 << 30;
    q->budget = q->cfg.hbm_budget_bytes ? q->cfg.hbm_budget_bytes : (free_b > reserve ? free_b - reserve : 0);
  } else {
    q->budget = q->cfg.hbm_budget_bytes ? q->cfg.hbm_budget_bytes : ((size_t)1 << 40);
  }
  q->st.hbm_budget = q->budget;
  if (const char* path = std::getenv("SENSE_QUEUE_LOG")) {
    if (*path) {
      q->log = std::fopen(path, "a");
      if (!q->log) {
        if (!q->hooks.fake_device) {
          cudaEventDestroy(q->admitted);
          cudaStreamDestroy(q->stream);
        }
        delete q;
        return qfail(SENSE_EINVAL, std::string("cannot open SENSE_QUEUE_LOG file ") + path);
      }
    }
  }
  q->worker = std::thread(worker_main, q);
  *out = q;
  return SENSE_OK;
}

sense_status sense_queue_submit(sense_queue* q, const sense_shape* shape, const void* y_host, const void* S_host,
                                const int32_t* lines_host, int max_iter, double rel_tol, uint64_t* req_id) {
  sense::TraceRange trace_range("sense_queue_submit");
  if (!q || !shape || !y_host || !S_host || !lines_host || !req_id)
    return qfail(SENSE_EINVAL, "queue, shape, inputs and req_id are required");
  const sense_shape& sh = *shape;
  if (sh.frames < 1 || sh.coils < 1 || sh.lines < 1 || sh.lines > sh.ny || max_iter < 1 || !(rel_tol >= 0.0))
    return qfail(SENSE_EINVAL, "bad shape, max_iter or rel_tol");
  if (sh.storage != SENSE_STORE_C64 && sh.storage != SENSE_STORE_BF16) return qfail(SENSE_EINVAL, "bad storage");
  if (sh.centred != 0 && sh.centred != 1) return qfail(SENSE_EINVAL, "centred must be 0 or 1");
  if (!sense_size_supported(sh.ny) || !sense_size_supported(sh.nx))
    return qfail(SENSE_EUNSUPPORTED_SIZE, "no compiled transform for this ny / nx");
  const Clock::time_point t_arrive = Clock::now();  // latency counts the staging copy
  Request* r = new Request();
  r->sh = sh;
  r->max_iter = max_iter;
  r->tol = rel_tol;
  r->need = request_need(sh);
  const size_t F = sh.frames, img = (size_t)sh.ny * sh.nx, e = elem_bytes(sh.storage);
  r->y_bytes = F * sh.coils * sh.lines * sh.nx * e;
  r->s_bytes = (size_t)sh.coils * img * e;
  r->l_bytes = F * sh.lines * sizeof(int);
  r->x_bytes = F * img * sizeof(float2);
  {
    std::lock_guard<std::mutex> lock(q->mu);
    q->st.submitted++;
    if (r->need > q->budget) {
      q->st.refused++;
      delete r;
      return qfail(SENSE_EQUEUE_FULL, "request needs more device memory than the queue's budget");
    }
  }
  PinnedArena& ar = *q->arena;
  r->y_h = ar.get(r->y_bytes);
  r->s_h = ar.get(r->s_bytes);
  r->lines_h = static_cast<int*>(ar.get(r->l_bytes));
  r->x_h = static_cast<float2*>(ar.get(r->x_bytes));
  r->iters_h = static_cast<int*>(ar.get(sizeof(int) * F));
  r->outcome_h = static_cast<int*>(ar.get(sizeof(int) * F));
  r->resid_h = static_cast<double*>(ar.get(sizeof(double) * F));
  r->err_h = static_cast<int*>(ar.get(sizeof(int)));
  if (!(r->y_h && r->s_h && r->lines_h && r->x_h && r->iters_h && r->outcome_h && r->resid_h && r->err_h)) {
    free_host(q, r);
    free_outputs(q, r);
    delete r;
    return qfail(SENSE_ENOMEM, "pinned staging allocation failed");
  }
  *r->err_h = 0;
  parallel_copy(r->y_h, y_host, r->y_bytes);
  parallel_copy(r->s_h, S_host, r->s_bytes);
  memcpy(r->lines_h, lines_host, r->l_bytes);
  r->t_submit = t_arrive;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    r->id = q->next_id++;
    q->reqs[r->id] = r;
    q->pending.push_back(r);
    *req_id = r->id;
    if (q->any_submit) {
      const double gap = std::chrono::duration<double, std::milli>(t_arrive - q->last_submit).count();
      q->gap_ms = q->gap_ms > 0.0 ? 0.75 * q->gap_ms + 0.25 * gap : gap;
    }
    q->any_submit = true;
    q->last_submit = t_arrive;
  }
  q->cv_work.notify_all();
  return SENSE_OK;
}

sense_status sense_queue_poll(sense_queue* q, uint64_t id, int* state, int* iters) {
  if (!q) return qfail(SENSE_EINVAL, "queue is NULL");
  std::lock_guard<std::mutex> lock(q->mu);
  auto it = q->reqs.find(id);
  if (it == q->reqs.end()) return qfail(SENSE_ENOTFOUND, "unknown request id");
  if (state) *state = it->second->state;
  if (iters) *iters = it->second->ticks;
  return SENSE_OK;
}

sense_status sense_queue_wait(sense_queue* q, uint64_t id, sense_c32* x_host, int32_t* iters_host, double* resid_host,
                              int32_t* outcome_host, double timeout_s) {
  sense::TraceRange trace_range("sense_queue_wait");
  if (!q) return qfail(SENSE_EINVAL, "queue is NULL");
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lock(q->mu);
    auto it = q->reqs.find(id);
    if (it == q->reqs.end()) return qfail(SENSE_ENOTFOUND, "unknown request id");
    r = it->second;
    auto finished = [&] { return r->state >= SENSE_REQ_DONE; };
    if (timeout_s > 0) {
      if (!q->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), finished))
        return qfail(SENSE_ETIMEOUT, "request not finished within the timeout");
    } else {
      q->cv_done.wait(lock, finished);
    }
    q->reqs.erase(it);
  }
  sense_status rc = SENSE_OK;
  if (r->state == SENSE_REQ_DONE) {
    const size_t F = r->sh.frames;
    if (x_host) memcpy(x_host, r->x_h, r->x_bytes);
    if (iters_host) memcpy(iters_host, r->iters_h, sizeof(int) * F);
    if (resid_host) memcpy(resid_host, r->resid_h, sizeof(double) * F);
    if (outcome_host) memcpy(outcome_host, r->outcome_h, sizeof(int) * F);
    // a frame that broke down with a non-finite residual saw NaN or Inf values
    for (size_t f = 0; f < F; ++f)
      if (r->outcome_h[f] == SENSE_CG_BREAKDOWN && !std::isfinite(r->resid_h[f])) {
        rc = qfail(SENSE_ENUMERIC, "frame " + std::to_string(f) +
                                       ": non-finite CG values (NaN or Inf in y or S); outputs were copied");
        break;
      }
  } else if (r->state == SENSE_REQ_CANCELLED) {
    rc = qfail(SENSE_EINVAL, "request was cancelled");
  } else {
    rc = qfail(r->fail_status, r->fail_msg);
  }
  free_outputs(q, r);
  free_host(q, r);
  delete r;
  return rc;
}

sense_status sense_queue_cancel(sense_queue* q, uint64_t id) {
  if (!q) return qfail(SENSE_EINVAL, "queue is NULL");
  {
    std::lock_guard<std::mutex> lock(q->mu);
    auto it = q->reqs.find(id);
    if (it == q->reqs.end()) return qfail(SENSE_ENOTFOUND, "unknown request id");
    it->second->cancel = true;
  }
  q->cv_work.notify_all();
  return SENSE_OK;
}

sense_status sense_queue_stats_get(sense_queue* q, sense_queue_stats* out) {
  if (!q || !out) return qfail(SENSE_EINVAL, "queue and out are required");
  std::lock_guard<std::mutex> lock(q->mu);
  *out = q->st;
  out->p50_ms = percentile(q->lat_ms, 0.50);
  out->p99_ms = percentile(q->lat_ms, 0.99);
  double sum = 0.0, mx = 0.0;
  for (double v : q->lat_ms) {
    sum += v;
    mx = std::max(mx, v);
  }
  out->mean_ms = q->lat_ms.empty() ? 0.0 : sum / q->lat_ms.size();
  out->max_ms = mx;
  out->hbm_in_use = q->in_use;
  out->hbm_budget = q->budget;
  int running = 0;
  for (auto& kv : q->reqs)
    if (kv.second->state == SENSE_REQ_RUNNING) ++running;
  out->live = running;
  out->pending = (int)q->pending.size();
  out->staging_reserved = q->arena->reserved();
  out->staging_in_use = q->arena->in_use();
  return SENSE_OK;
}

sense_status sense_queue_set_variant(sense_queue* q, int ny, int nx, int storage, int variant) {
  if (!q) return qfail(SENSE_EINVAL, "queue is NULL");
  if (!sense_size_supported(ny) || !sense_size_supported(nx))
    return qfail(SENSE_EUNSUPPORTED_SIZE, "no compiled transform for this ny / nx");
  if (storage != SENSE_STORE_C64 && storage != SENSE_STORE_BF16) return qfail(SENSE_EINVAL, "bad storage");
  if (variant < 0 || variant >= kNormVariants || normal_variant_width(ny, variant) <= 0)
    return qfail(SENSE_EINVAL, "no such normal-operator variant for this ny");
  std::lock_guard<std::mutex> lock(q->mu);
  const auto key = std::make_tuple(ny, nx, storage);
  auto it = q->variants.find(key);
  if (it != q->variants.end() && it->second != variant)
    return qfail(SENSE_EINVAL, "the size class already runs another variant (set it before its first request)");
  q->variants[key] = variant;
  return SENSE_OK;
}

int sense_queue_variant(sense_queue* q, int ny, int nx, int storage) {
  if (!q) return -1;
  std::lock_guard<std::mutex> lock(q->mu);
  auto it = q->variants.find(std::make_tuple(ny, nx, storage));
  return it == q->variants.end() ? -1 : it->second;
}

sense_status sense_queue_destroy(sense_queue* q) {
  if (!q) return SENSE_OK;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    q->stop = true;
    for (Request* r : q->pending) {
      r->state = SENSE_REQ_CANCELLED;
      r->t_done = Clock::now();
      q->st.cancelled++;
      log_request(q, r);
    }
  }
  q->cv_work.notify_all();
  if (q->worker.joinable()) q->worker.join();
  for (auto& kv : q->reqs) {
    Request* r = kv.second;
    if (!q->hooks.fake_device) free_device(r, q->stream);
    free_outputs(q, r);
    free_host(q, r);
    delete r;
  }
  if (!q->hooks.fake_device) {
    for (auto& kv : q->classes) {
      SizeClass& c = kv.second;
      for (void* p : {(void*)c.ints, (void*)c.part_nrm, (void*)c.part_upd, (void*)c.table_d, (void*)c.status_d})
        if (p) cudaFree(p);
      if (c.table_h) cudaFreeHost(c.table_h);
      if (c.status_h) cudaFreeHost(c.status_h);
      if (c.stream) {
        cudaStreamSynchronize(c.stream);
        cudaStreamDestroy(c.stream);
      }
      if (c.done) cudaEventDestroy(c.done);
    }
    for (auto& kv : q->twiddles) cudaFree(kv.second);
    if (q->admitted) cudaEventDestroy(q->admitted);
    if (q->stream) {
      cudaStreamSynchronize(q->stream);
      cudaStreamDestroy(q->stream);
    }
  }
  if (q->log) std::fclose(q->log);
  q->arena.reset();  // after the stream is idle: no copy still reads or writes staging
  delete q;
  return SENSE_OK;
}

}  // extern "C"
