// Private definition of the plan object and the host helpers shared by the
// library's units (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "persistent.cuh"
#include "sense.h"

using sense::CgState;
using sense::PFrame;

struct sense_plan {
  sense_shape sh{};
  int device = 0;
  int tiles = 0;        // column tiles per frame (adjoint / forward column passes)
  int norm_variant = 0;  // kernel variant of the normal operator (autotuned)
  int norm_tiles = 0;    // column tiles per frame of that variant
  int cg_mode = 1;       // 0: per-phase kernels replayed as CUDA graphs; 1: one persistent launch
  int col_tma = 1;       // 1: TMA column passes; 2: single-launch fused E / E^H (square, TMA lengths); 0: per-tile
  int cg_order = -2;     // persistent CG item order (kOrderAuto; a test hook can pin another, see sense_testing.h)
  int* fused_ints = nullptr;  // ticket and per-frame counters of the fused operators ([F + 1])
  int tiles8 = 0;        // 8-column tiles per frame (TMA column passes)
  double lambda = 0.0;   // Tikhonov weight of CG: (E^H E + lambda I) x = E^H y
  double lambda_t = 0.0; // temporal weight: > 0 couples the frames into one CG (persistent mode)
  cudaStream_t pool = nullptr;  // non-null: workspace is stream-ordered (cudaMallocAsync) on this stream
  CUtensorMap tmap_host;        // TMA descriptor of the maps S for the persistent kernel
  CUtensorMap* tmap_d = nullptr;
  const void* tmap_S = nullptr; // S and tile width the descriptor was encoded for
  int tmap_W = 0;
  bool own_tw = true;           // false: twiddle tables are shared and owned elsewhere
  int sms = 0;           // multiprocessors of the plan's device
  PFrame* ptable = nullptr;       // device frame table of the persistent kernel
  PFrame* ptable_host = nullptr;  // pinned staging copy
  const void* ptable_key[3] = {nullptr, nullptr, nullptr};  // S, lines, x the table was built for
  double ptable_tol = -1.0;
  int* pints = nullptr;           // nrm_arrive, upd_arrive, nrm_ready, upd_ready ([4][F]), ticket
  double* part_nrm = nullptr;     // [F][max tiles]
  double* part_upd = nullptr;     // [F][max chunks]
  int max_chunks = 0;
  int upd_blocks = 0;   // CG-update blocks per frame
  size_t img = 0;       // ny * nx
  float2* tw_y = nullptr;
  float2* tw_x = nullptr;
  float2* tmp = nullptr;  // [F][C][L][nx] intermediate of E / E^H
  float2* r = nullptr;
  float2* pp[2] = {nullptr, nullptr};  // search directions, ping-pong between iterations
  float2* q = nullptr;
  void* maps_t = nullptr;  // S^T [C][nx][ny] for variants with lane-major tiles (allocated on first use)
  // device copies of the host buffers of sense_cg_solve_host (allocated on its first call)
  void* hio_y = nullptr;
  void* hio_S = nullptr;
  int* hio_lines = nullptr;
  float2* hio_x = nullptr;
  int* hio_ints = nullptr;      // iterations, outcomes ([2][F])
  double* hio_resid = nullptr;  // [F]

  double* dbl = nullptr;  // rho, rho0, alpha, beta, resid  ([5][F])
  int* ints = nullptr;    // iters, outcome, active ([3][F]), live, err
  unsigned* counter = nullptr;
  double* part = nullptr;
  int part_stride = 0;
  int* live_host = nullptr;  // pinned
  size_t ws_bytes = 0;
  std::vector<void*> allocs;
  cudaStream_t capture_stream = nullptr;
  // kernel timers (diagnostic mode): event pairs per launch, summed per phase
  int timing = 0;
  double phase_ms[SENSE_PHASE_COUNT] = {};
  long phase_launches[SENSE_PHASE_COUNT] = {};
  struct Span { int phase; cudaEvent_t a, b; };
  std::vector<Span> pending;
  // CUDA graphs of the CG iteration loop, keyed by the arguments they bake in
  std::map<std::tuple<const void*, const void*, const void*, int, int, double>, cudaGraphExec_t> graphs;

  CgState cg(double tol) const {
    CgState g;
    const int F = sh.frames;
    g.rho = dbl;
    g.rho0 = dbl + F;
    g.alpha = dbl + 2 * F;
    g.beta = dbl + 3 * F;
    g.resid = dbl + 4 * F;
    g.iters = ints;
    g.outcome = ints + F;
    g.active = ints + 2 * F;
    g.live = ints + 3 * F;
    g.counter = counter;
    g.part = part;
    g.part_stride = part_stride;
    g.tol = tol;
    return g;
  }
  int* err() const { return ints + 3 * sh.frames + 1; }
};

namespace sense {

// Stores the message sense_last_error() returns on this thread.
void record_error(const std::string& msg);

// CG start for a plan: b = E^H y into r and p_0, x = 0, per-frame scalars
// (rho0, active, ...), asynchronously on `st`.
sense_status plan_cg_start(sense_plan* pl, const void* y, const void* S, const int* lines, float2* x, double tol,
                           cudaStream_t st);

// Frame-table entries of a plan's frames for the persistent CG kernel;
// `base` is the table index of the plan's first frame.
void plan_frames(const sense_plan* pl, const void* S, const int* lines, float2* x, int k0, double tol,
                 PFrame* out, int base);

// A plan whose workspace comes from the device's stream-ordered pool on `st`
// and whose twiddle tables are the caller's (shared per size): no device-wide
// synchronisation on creation or destruction.  For request-scoped plans.
sense_status plan_create_pooled(const sense_shape* shape, int device, cudaStream_t st, const float2* tw_y,
                                const float2* tw_x, sense_plan** out);
void plan_destroy_pooled(sense_plan* pl);
// Select the normal-operator variant without synchronising (the plan has no
// captured graphs).
sense_status plan_set_variant_nosync(sense_plan* pl, int variant);
// exp(-2 pi i m / n), m < n, in FP64 rounded once to FP32 (host table).
std::vector<float2> plan_twiddles(int n);

// Encode (when S or the kernel variant changed) the TMA descriptor of S and
// queue its upload on `st`.  Must not run during stream capture.
sense_status plan_prepare_tmap(sense_plan* pl, const void* S, cudaStream_t st);

// Maps read by the normal-operator tiles of the plan's current variant:
// plan_maps_buffer allocates S^T on first use if the variant reads it (not
// during stream capture); plan_maps then returns S itself, or S^T refreshed
// from S by a transpose queued on `st` (capturable once the buffer exists).
sense_status plan_maps_buffer(sense_plan* pl);
sense_status plan_maps(sense_plan* pl, const void* S, cudaStream_t st, const void** out);
bool plan_maps_transposed(const sense_plan* pl);

// Centred plans: map a finished CG solution x (all frames) from the
// modulated space the iterations run in back to the image, on `st`.
sense_status plan_centred_output(sense_plan* pl, float2* x, cudaStream_t st);

// Per-frame outputs of a finished CG solve of a plan (iterations, residual,
// outcome; NULL outputs are skipped).
sense_status plan_cg_finish(sense_plan* pl, int* iters_out, double* resid_out, int* outcome_out, cudaStream_t st);

}  // namespace sense
