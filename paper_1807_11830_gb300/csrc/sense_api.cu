// Host runtime and C ABI of libsense.so: plans (twiddles + workspace), the
// operator entry points and the CG-SENSE driver loop (captured once per
// argument set into a CUDA graph and replayed).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cg_kernels.cuh"
#include "colpass.cuh"
#include "fused.cuh"
#include "launch.h"
#include "plan.h"
#include "trace.h"
#include "sense.h"
#include "sense_testing.h"

using namespace sense;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace sense {
// Lets other units of the library report through sense_last_error().
void record_error(const std::string& msg) { g_last_error = msg; }
}  // namespace sense

namespace {

sense_status fail(sense_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define SENSE_CUDA_TRY(expr)                                                                  \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(SENSE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool aligned16(const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned4(const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map of `rows` rows of `cols` elements (4 or 8 bytes each, rows
// contiguous) with a box of box_cols x box_rows elements; a pure host
// computation (no device work), so it may run during stream capture.
bool encode_rows_2d(CUtensorMap* m, const void* base, int elem_bytes, size_t cols, size_t rows, int box_cols,
                    int box_rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 2,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of the TMA column passes: S [coils * ny] rows of nx, box 8 x (ny or ny / 2).
bool encode_maps_col(CUtensorMap* m, const sense_shape& sh, const void* S) {
  return encode_rows_2d(m, S, sh.storage == SENSE_STORE_BF16 ? 4 : 8, (size_t)sh.nx, (size_t)sh.coils * sh.ny, 8,
                        sh.ny <= 256 ? sh.ny : sh.ny / 2);
}

// exp(-2 pi i m / n), m = 0..n-1, in FP64 and rounded once to FP32.
std::vector<float2> twiddles(int n) {
  std::vector<float2> t((size_t)n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double a = -two_pi * (double)m / (double)n;
    t[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return t;
}

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

}  // namespace


namespace {

// Brackets one launch with a pair of events on `st` when the plan's timers
// are on.
class PhaseScope {
 public:
  PhaseScope(sense_plan* pl, int phase, cudaStream_t st) : pl_(pl), st_(st) {
    if (!pl->timing) return;
    span_.phase = phase;
    if (cudaEventCreate(&span_.a) != cudaSuccess || cudaEventCreate(&span_.b) != cudaSuccess) return;
    cudaEventRecord(span_.a, st_);
    on_ = true;
  }
  ~PhaseScope() {
    if (!on_) return;
    cudaEventRecord(span_.b, st_);
    pl_->pending.push_back(span_);
  }

 private:
  sense_plan* pl_;
  cudaStream_t st_;
  sense_plan::Span span_{};
  bool on_ = false;
};

void collect_spans(sense_plan* pl) {
  for (auto& sp : pl->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(sp.b) == cudaSuccess && cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
      pl->phase_ms[sp.phase] += ms;
      pl->phase_launches[sp.phase] += 1;
    }
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  pl->pending.clear();
}

template <class T>
sense_status dalloc(sense_plan* pl, T** out, size_t count) {
  void* ptr = nullptr;
  const size_t bytes = count * sizeof(T);
  cudaError_t e = pl->pool ? cudaMallocAsync(&ptr, bytes ? bytes : 16, pl->pool) : cudaMalloc(&ptr, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SENSE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  pl->allocs.push_back(ptr);
  pl->ws_bytes += bytes;
  *out = static_cast<T*>(ptr);
  return SENSE_OK;
}

}  // namespace

namespace sense {

bool plan_maps_transposed(const sense_plan* pl) {
  return normal_variant_transposed(pl->sh.ny, pl->norm_variant) != 0;
}

sense_status plan_maps_buffer(sense_plan* pl) {
  if (!plan_maps_transposed(pl) || pl->maps_t) return SENSE_OK;
  const size_t count = (size_t)pl->sh.coils * pl->img;
  sense_status rc;
  if (pl->sh.storage == SENSE_STORE_BF16) {
    __nv_bfloat162* ptr = nullptr;
    rc = dalloc(pl, &ptr, count);
    pl->maps_t = ptr;
  } else {
    float2* ptr = nullptr;
    rc = dalloc(pl, &ptr, count);
    pl->maps_t = ptr;
  }
  return rc;
}

sense_status plan_maps(sense_plan* pl, const void* S, cudaStream_t st, const void** out) {
  *out = S;
  if (!plan_maps_transposed(pl)) return SENSE_OK;
  sense_status rc = plan_maps_buffer(pl);
  if (rc != SENSE_OK) return rc;
  const sense_shape& sh = pl->sh;
  PhaseScope ps(pl, SENSE_PHASE_MAPS_TRANSPOSE, st);
  const cudaError_t e = launch_transpose_maps(sh.storage == SENSE_STORE_BF16, S, pl->maps_t, sh.ny, sh.nx, sh.coils, st);
  if (e != cudaSuccess) return fail(SENSE_ECUDA, std::string("map transpose: ") + cudaGetErrorString(e));
  *out = pl->maps_t;
  return SENSE_OK;
}

sense_status plan_centred_output(sense_plan* pl, float2* x, cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  if (!sh.centred) return SENSE_OK;
  const long n = (long)sh.frames * (long)pl->img;
  k_checkerboard<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, sh.ny, sh.nx, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SENSE_ECUDA, std::string("centred output: ") + cudaGetErrorString(e));
  return SENSE_OK;
}

}  // namespace sense

namespace {

void release(sense_plan* pl) {
  collect_spans(pl);
  for (auto& kv : pl->graphs) cudaGraphExecDestroy(kv.second);
  pl->graphs.clear();
  for (void* ptr : pl->allocs) {
    if (pl->pool)
      cudaFreeAsync(ptr, pl->pool);
    else
      cudaFree(ptr);
  }
  pl->allocs.clear();
  if (pl->live_host) cudaFreeHost(pl->live_host);
  pl->live_host = nullptr;
  if (pl->ptable_host) cudaFreeHost(pl->ptable_host);
  pl->ptable_host = nullptr;
  if (pl->capture_stream) cudaStreamDestroy(pl->capture_stream);
  pl->capture_stream = nullptr;
}

sense_status check_shape(const sense_shape* sh) {
  if (!sh) return fail(SENSE_EINVAL, "shape is NULL");
  if (sh->frames < 1 || sh->coils < 1 || sh->ny < 1 || sh->nx < 1)
    return fail(SENSE_EINVAL, "frames, coils, ny and nx must be >= 1");
  if (sh->frames > 65535) return fail(SENSE_EINVAL, "at most 65535 frames per plan");
  if (sh->lines < 1 || sh->lines > sh->ny) return fail(SENSE_EINVAL, "lines must be in [1, ny]");
  if (sh->storage != SENSE_STORE_C64 && sh->storage != SENSE_STORE_BF16)
    return fail(SENSE_EINVAL, "storage must be SENSE_STORE_C64 or SENSE_STORE_BF16");
  if (!size_supported(sh->ny) || !size_supported(sh->nx))
    return fail(SENSE_EUNSUPPORTED_SIZE, "no compiled transform for ny=" + std::to_string(sh->ny) +
                                             " / nx=" + std::to_string(sh->nx));
  if (sh->centred != 0 && sh->centred != 1) return fail(SENSE_EINVAL, "centred must be 0 or 1");
  return SENSE_OK;
}

// (-1)^(ny/2 + nx/2): the constant of the centred 2D transform
float centred_sign(const sense_shape& sh) { return ((sh.ny / 2 + sh.nx / 2) & 1) ? -1.0f : 1.0f; }

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

sense_status launch_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SENSE_OK;
  return fail(SENSE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- operator launch sequences (shared by the entry points and graph capture) ----

template <class St>
sense_status run_forward(sense_plan* pl, const float2* x, const void* S, const int* lines, void* y,
                         cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  FwdColArgs<St> a{};
  a.x = x;
  a.S = static_cast<const typename St::T*>(S);
  a.lines = lines;
  a.tmp = pl->tmp;
  a.tw = pl->tw_y;
  a.nx = sh.nx;
  a.coils = sh.coils;
  a.L = sh.lines;
  a.centred = sh.centred;
  a.err = pl->err();
  sense_status rc;
  if (pl->col_tma == 2 && sh.ny == sh.nx && coltma_supported(sh.ny)) {  // both passes in one launch
    CUtensorMap tmS;
    if (encode_maps_col(&tmS, sh, S)) {
      const int row_items = ((sh.coils * sh.lines + 7) / 8 + kFusedRowTiles - 1) / kFusedRowTiles;
      FusedSched sc{reinterpret_cast<unsigned*>(pl->fused_ints + sh.frames), pl->fused_ints, sh.frames, pl->tiles8,
                    row_items, kFusedLag};
      SENSE_CUDA_TRY(cudaMemsetAsync(pl->fused_ints, 0, sizeof(int) * ((size_t)sh.frames + 1), st));
      PhaseScope ps(pl, SENSE_PHASE_FWD_FUSED, st);
      const cudaError_t e = launch_forward_fused<St>(sh.ny, tmS, a, y, sc, centred_sign(sh), pl->sms, st);
      if (e != cudaErrorNotSupported) return launch_status(e, "fused forward operator");
    }
  }
  {
    PhaseScope ps(pl, SENSE_PHASE_FWD_COL, st);
    cudaError_t e = cudaErrorNotSupported;
    CUtensorMap tmS;
    if (pl->col_tma && coltma_supported(sh.ny) && encode_maps_col(&tmS, sh, S))
      e = launch_fwd_col_tma<St>(sh.ny, tmS, a, pl->tiles8, sh.frames, pl->sms, st);
    if (e == cudaErrorNotSupported) e = launch_fwd_col<St>(sh.ny, a, pl->tiles, sh.frames, st);
    rc = launch_status(e, "forward column pass");
  }
  if (rc != SENSE_OK) return rc;
  RowArgs<float2, typename St::T> ra{};
  ra.in = pl->tmp;
  ra.out = static_cast<typename St::T*>(y);
  ra.tw = pl->tw_x;
  ra.rows = (long)sh.frames * sh.coils * sh.lines;
  ra.centred = sh.centred;
  ra.cs = centred_sign(sh);
  ra.err = pl->err();
  PhaseScope ps(pl, SENSE_PHASE_ROWS_FWD, st);
  return launch_status(launch_rows_fwd<St>(sh.nx, ra, st), "forward row pass");
}

template <class St>
sense_status run_rows_inv(sense_plan* pl, const void* y, cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  RowArgs<typename St::T, float2> ra{};
  ra.in = static_cast<const typename St::T*>(y);
  ra.out = pl->tmp;
  ra.tw = pl->tw_x;
  ra.rows = (long)sh.frames * sh.coils * sh.lines;
  ra.centred = sh.centred;
  ra.cs = centred_sign(sh);
  ra.err = pl->err();
  PhaseScope ps(pl, SENSE_PHASE_ROWS_INV, st);
  return launch_status(launch_rows_inv<St>(sh.nx, ra, st), "adjoint row pass");
}

template <class St>
sense_status run_adjoint(sense_plan* pl, int mode, const void* y, const void* S, const int* lines, float2* x,
                         float* rss, double tol, cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  if (pl->col_tma == 2 && sh.ny == sh.nx && coltma_supported(sh.ny)) {  // both passes in one launch
    CUtensorMap tmK, tmS;
    const bool maps_ok =
        encode_rows_2d(&tmK, pl->tmp, 8, (size_t)sh.nx, (size_t)sh.frames * sh.coils * sh.lines, 8,
                       kbox_rows(sh.lines)) &&
        (mode == 2 ? encode_rows_2d(&tmS, pl->tmp, 8, (size_t)sh.nx, 1, 8, 1) : encode_maps_col(&tmS, sh, S));
    if (maps_ok) {
      const int row_items = ((sh.coils * sh.lines + 7) / 8 + kFusedRowTiles - 1) / kFusedRowTiles;
      FusedSched sc{reinterpret_cast<unsigned*>(pl->fused_ints + sh.frames), pl->fused_ints, sh.frames, row_items,
                    pl->tiles8, kFusedLag};
      SENSE_CUDA_TRY(cudaMemsetAsync(pl->fused_ints, 0, sizeof(int) * ((size_t)sh.frames + 1), st));
      const bool ybf16 = sh.storage == SENSE_STORE_BF16;
      cudaError_t e;
      PhaseScope ps(pl, SENSE_PHASE_ADJ_FUSED, st);
      if (mode == 2) {
        AdjColArgs<StC64> a{};
        a.tmp = pl->tmp;
        a.lines = lines;
        a.tw = pl->tw_y;
        a.rss = rss;
        a.nx = sh.nx;
        a.coils = sh.coils;
        a.L = sh.lines;
        a.tiles = pl->tiles8;
        a.centred = sh.centred;
        a.err = pl->err();
        e = launch_adjoint_fused<StC64>(sh.ny, 2, ybf16, tmK, tmS, a, y, pl->tmp, sc, centred_sign(sh), pl->sms, st);
      } else {
        AdjColArgs<St> a{};
        a.tmp = pl->tmp;
        a.S = static_cast<const typename St::T*>(S);
        a.lines = lines;
        a.tw = pl->tw_y;
        a.x = x;
        a.r = pl->r;
        a.p = pl->pp[0];
        a.nx = sh.nx;
        a.coils = sh.coils;
        a.L = sh.lines;
        a.tiles = pl->tiles8;
        a.centred = sh.centred;
        a.err = pl->err();
        a.cg = pl->cg(tol);
        e = launch_adjoint_fused<St>(sh.ny, mode, ybf16, tmK, tmS, a, y, pl->tmp, sc, centred_sign(sh), pl->sms, st);
      }
      if (e != cudaErrorNotSupported) return launch_status(e, "fused adjoint operator");
    }
  }
  sense_status rc = run_rows_inv<St>(pl, y, st);
  if (rc != SENSE_OK) return rc;
  // TMA column passes: the intermediate [F*C*L][nx] as a tensor map (box 8 x rows per box)
  CUtensorMap tmK, tmS;
  const bool tma = pl->col_tma && coltma_supported(sh.ny) &&
                   encode_rows_2d(&tmK, pl->tmp, 8, (size_t)sh.nx, (size_t)sh.frames * sh.coils * sh.lines, 8,
                                  kbox_rows(sh.lines)) &&
                   (mode == 2 ? encode_rows_2d(&tmS, pl->tmp, 8, (size_t)sh.nx, 1, 8, 1) : encode_maps_col(&tmS, sh, S));
  if (mode == 2) {
    AdjColArgs<StC64> a{};
    a.tmp = pl->tmp;
    a.lines = lines;
    a.tw = pl->tw_y;
    a.rss = rss;
    a.nx = sh.nx;
    a.coils = sh.coils;
    a.L = sh.lines;
    a.tiles = pl->tiles;
    a.centred = sh.centred;
    a.err = pl->err();
    PhaseScope ps(pl, SENSE_PHASE_ADJ_COL, st);
    cudaError_t e = cudaErrorNotSupported;
    if (tma) {
      a.tiles = pl->tiles8;
      e = launch_adj_col_tma<StC64>(sh.ny, 2, tmK, tmS, a, sh.frames, pl->sms, st);
      a.tiles = pl->tiles;
    }
    if (e == cudaErrorNotSupported) e = launch_adj_col<StC64>(sh.ny, 2, a, pl->tiles, sh.frames, st);
    return launch_status(e, "rss column pass");
  }
  AdjColArgs<St> a{};
  a.tmp = pl->tmp;
  a.S = static_cast<const typename St::T*>(S);
  a.lines = lines;
  a.tw = pl->tw_y;
  a.x = x;
  a.r = pl->r;
  a.p = pl->pp[0];
  a.nx = sh.nx;
  a.coils = sh.coils;
  a.L = sh.lines;
  a.tiles = pl->tiles;
  a.centred = sh.centred;  // mode 1 (CG start) works in the modulated space: no image signs there
  a.err = pl->err();
  a.cg = pl->cg(tol);
  PhaseScope ps(pl, SENSE_PHASE_ADJ_COL, st);
  cudaError_t e = cudaErrorNotSupported;
  if (tma) {
    a.tiles = pl->tiles8;
    e = launch_adj_col_tma<St>(sh.ny, mode, tmK, tmS, a, sh.frames, pl->sms, st);
    a.tiles = pl->tiles;
  }
  if (e == cudaErrorNotSupported) e = launch_adj_col<St>(sh.ny, mode, a, pl->tiles, sh.frames, st);
  return launch_status(e, "adjoint column pass");
}

template <class St>
sense_status run_normal(sense_plan* pl, const float2* x, const void* S, const int* lines, float2* out,
                        cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  const void* maps = nullptr;
  sense_status rc = plan_maps(pl, S, st, &maps);
  if (rc != SENSE_OK) return rc;
  NormalArgs<St> a{};
  a.x = x;
  a.out = out;
  a.S = static_cast<const typename St::T*>(maps);
  a.lines = lines;
  a.tw = pl->tw_y;
  a.nx = sh.nx;
  a.coils = sh.coils;
  a.L = sh.lines;
  a.tiles = pl->norm_tiles;
  a.centred = sh.centred;
  a.err = pl->err();
  PhaseScope ps(pl, SENSE_PHASE_NORMAL, st);
  return launch_status(launch_normal<St>(sh.ny, pl->norm_variant, false, a, sh.frames, st), "normal operator");
}

// Iteration k of CG: q = E^H E p_k (p_k = r + beta p_{k-1} formed on the fly
// for k > 0), alpha; then x += alpha p_k, r -= alpha q, beta / stopping test.
// p_k lives in pp[k & 1]; p_0 = r_0 is written by the CG start into pp[0].
template <class St>
sense_status run_cg_iteration(sense_plan* pl, const void* S, const int* lines, float2* x, int k, double tol,
                              cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  const int p_update = k > 0 ? 1 : 0;
  float2* p_cur = pl->pp[k & 1];
  NormalArgs<St> a{};
  a.p_src = p_update ? pl->pp[(k - 1) & 1] : p_cur;
  a.p_dst = p_cur;
  a.r = pl->r;
  a.q = pl->q;
  a.S = static_cast<const typename St::T*>(S);
  a.lines = lines;
  a.tw = pl->tw_y;
  a.nx = sh.nx;
  a.coils = sh.coils;
  a.L = sh.lines;
  a.tiles = pl->norm_tiles;
  a.p_update = p_update;
  a.lambda = (float)pl->lambda;
  a.err = pl->err();
  a.cg = pl->cg(tol);
  sense_status rc;
  {
    PhaseScope ps(pl, SENSE_PHASE_CG_NORMAL, st);
    rc = launch_status(launch_normal<St>(sh.ny, pl->norm_variant, true, a, sh.frames, st), "CG normal pass");
  }
  if (rc != SENSE_OK) return rc;
  UpdateArgs u{};
  u.x = reinterpret_cast<float4*>(x);
  u.p = reinterpret_cast<const float4*>(p_cur);
  u.q = reinterpret_cast<const float4*>(pl->q);
  u.r = reinterpret_cast<float4*>(pl->r);
  u.img4 = (long)(pl->img / 2);
  u.blocks_per_frame = pl->upd_blocks;
  u.cg = pl->cg(tol);
  PhaseScope ps(pl, SENSE_PHASE_CG_UPDATE, st);
  k_cg_update<<<dim3(pl->upd_blocks, sh.frames), UPD_THREADS, 0, st>>>(u);
  return launch_status(cudaGetLastError(), "CG update");
}

template <class St>
sense_status run_cg_chunk(sense_plan* pl, const void* S, const int* lines, float2* x, int first, int count,
                          double tol, cudaStream_t st) {
  for (int i = 0; i < count; ++i) {
    sense_status rc = run_cg_iteration<St>(pl, S, lines, x, first + i, tol, st);
    if (rc != SENSE_OK) return rc;
  }
  return SENSE_OK;
}

// Replay (capturing on first use) the graph of `count` iterations starting at
// iteration `first` for these arguments.
template <class St>
sense_status cg_chunk_graph(sense_plan* pl, const void* S, const int* lines, float2* x, int first, int count,
                            double tol, cudaStream_t st) {
  if (pl->timing || pl->cg_mode == 2) return run_cg_chunk<St>(pl, S, lines, x, first, count, tol, st);
  const int first_key = first == 0 ? 0 : 1 + (first & 1);  // p_update and ping-pong parity
  auto key = std::make_tuple(S, (const void*)lines, (const void*)x, first_key, count, tol);
  auto it = pl->graphs.find(key);
  if (it == pl->graphs.end()) {
    cudaStream_t cs = pl->capture_stream;
    SENSE_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    sense_status rc = run_cg_chunk<St>(pl, S, lines, x, first, count, tol, cs);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (rc != SENSE_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ee != cudaSuccess) return fail(SENSE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    cudaGraphExec_t exec = nullptr;
    ee = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ee != cudaSuccess) return fail(SENSE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ee));
    if (pl->graphs.size() > 64) {  // bound the cache
      for (auto& kv : pl->graphs) cudaGraphExecDestroy(kv.second);
      pl->graphs.clear();
    }
    it = pl->graphs.emplace(key, exec).first;
  }
  SENSE_CUDA_TRY(cudaGraphLaunch(it->second, st));
  return SENSE_OK;
}

// ---- autotune cache: in-process map, optionally mirrored to a text file ----
// (SENSE_AUTOTUNE_CACHE=path; one "device ny nx coils frames lines storage mode variant" per line,
// mode 1 for a persistent-CG timing, 0 for a normal-operator launch timing)
struct TuneKey {
  int device, ny, nx, coils, frames, lines, storage, mode;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, ny, nx, coils, frames, lines, storage, mode) <
           std::tie(o.device, o.ny, o.nx, o.coils, o.frames, o.lines, o.storage, o.mode);
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune;
bool g_tune_loaded = false;

void tune_load_file_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("SENSE_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return;
  TuneKey k{};
  int v = 0;
  while (std::fscanf(fh, "%d %d %d %d %d %d %d %d %d", &k.device, &k.ny, &k.nx, &k.coils, &k.frames, &k.lines,
                     &k.storage, &k.mode, &v) == 9)
    if (v >= 0 && v < kNormVariants && normal_variant_width(k.ny, v) > 0) g_tune[k] = v;
  std::fclose(fh);
}

int tune_cache_lookup(const TuneKey& k) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load_file_locked();
  auto it = g_tune.find(k);
  return it == g_tune.end() ? -1 : it->second;
}

void tune_cache_store(const TuneKey& k, int v) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load_file_locked();
  g_tune[k] = v;
  const char* path = std::getenv("SENSE_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%d %d %d %d %d %d %d %d %d\n", k.device, k.ny, k.nx, k.coils, k.frames, k.lines, k.storage,
               k.mode, v);
  std::fclose(fh);
}

constexpr int kPollEvery = 5;

// All CG iterations in one persistent launch (see persistent.cuh).
template <class St>
sense_status run_cg_persistent(sense_plan* pl, const void* S, const int* lines, float2* x, int max_iter, double tol,
                               cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  const int F = sh.frames;
  if (!plan_maps_transposed(pl)) {  // S here is what the tiles read: S, or S^T
    sense_status rc = plan_prepare_tmap(pl, S, st);
    if (rc != SENSE_OK) return rc;
  }
  if (pl->ptable_key[0] != S || pl->ptable_key[1] != (const void*)lines || pl->ptable_key[2] != (const void*)x ||
      pl->ptable_tol != tol) {
    SENSE_CUDA_TRY(cudaStreamSynchronize(st));  // the staging copy may still be read by an earlier call
    plan_frames(pl, S, lines, x, 0, tol, pl->ptable_host, 0);
    SENSE_CUDA_TRY(cudaMemcpyAsync(pl->ptable, pl->ptable_host, sizeof(PFrame) * F, cudaMemcpyHostToDevice, st));
    pl->ptable_key[0] = S;
    pl->ptable_key[1] = lines;
    pl->ptable_key[2] = x;
    pl->ptable_tol = tol;
  }
  SENSE_CUDA_TRY(cudaMemsetAsync(pl->pints, 0, sizeof(int) * (4 * (size_t)F + 1), st));
  const int threads = normal_variant_threads(sh.ny, pl->norm_variant);
  PArgs a{};
  a.frames = pl->ptable;
  a.nframes = F;
  a.nx = sh.nx;
  a.tiles = pl->norm_tiles;
  a.chunks = update_chunks(pl->img, threads);
  a.lag = persistent_order(pl->ptable_host, F);
  if (a.lag != kOrderIterationMajor) a.lag = pl->cg_order;  // frames coupled in time keep the iteration-major order
  a.iters = max_iter;
  a.ticket = reinterpret_cast<unsigned*>(pl->pints + 4 * F);
  a.tw = pl->tw_y;
  a.err = pl->err();
  a.st.nrm_arrive = reinterpret_cast<unsigned*>(pl->pints);
  a.st.upd_arrive = reinterpret_cast<unsigned*>(pl->pints + F);
  a.st.nrm_ready = pl->pints + 2 * F;
  a.st.upd_ready = pl->pints + 3 * F;
  a.st.part_nrm = pl->part_nrm;
  a.st.part_upd = pl->part_upd;
  if (a.chunks > pl->max_chunks) return fail(SENSE_EINVAL, "internal: update chunks exceed the workspace");
  PhaseScope ps(pl, SENSE_PHASE_CG_PERSISTENT, st);
  return launch_status(launch_cg_persistent<St>(sh.ny, pl->norm_variant, a, pl->sms, st), "persistent CG");
}

template <class St>
sense_status run_cg_solve(sense_plan* pl, const void* y, const void* S, const int* lines, int max_iter, double tol,
                          float2* x, int* iters_out, double* resid_out, int* outcome_out, cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  SENSE_CUDA_TRY(cudaMemsetAsync(pl->counter, 0, sizeof(unsigned) * sh.frames, st));
  SENSE_CUDA_TRY(cudaMemsetAsync(pl->cg(tol).live, 0, sizeof(int), st));
  sense_status rc = run_adjoint<St>(pl, 1, y, S, lines, x, nullptr, tol, st);
  if (rc != SENSE_OK) return rc;
  const void* maps = nullptr;  // what the normal-operator tiles read
  rc = plan_maps(pl, S, st, &maps);
  if (rc != SENSE_OK) return rc;
  const int coupled = pl->lambda_t > 0.0 ? 1 : 0;
  if (coupled) {  // one CG over all frames: the group's start scalars from the frames'
    k_cg_couple_start<<<1, 32, 0, st>>>(pl->cg(tol), sh.frames);
    rc = launch_status(cudaGetLastError(), "coupled CG start");
    if (rc != SENSE_OK) return rc;
  }
  if (pl->cg_mode == 1 || coupled) {  // frames coupled in time run in the persistent kernel only
    if (max_iter > 0) rc = run_cg_persistent<St>(pl, maps, lines, x, max_iter, tol, st);
    if (rc != SENSE_OK) return rc;
    rc = plan_centred_output(pl, x, st);
    if (rc != SENSE_OK) return rc;
    PhaseScope ps(pl, SENSE_PHASE_CG_FINISH, st);
    k_cg_finish<<<(sh.frames + 127) / 128, 128, 0, st>>>(pl->cg(tol), sh.frames, iters_out, resid_out, outcome_out,
                                                          coupled);
    return launch_status(cudaGetLastError(), "CG finish");
  }
  {  // kernel attributes are set outside stream capture
    NormalArgs<St> none{};
    rc = launch_status(launch_normal<St>(sh.ny, pl->norm_variant, true, none, 0, st), "CG normal set-up");
    if (rc != SENSE_OK) return rc;
  }
  if (tol <= 0.0) {
    if (max_iter > 0) rc = cg_chunk_graph<St>(pl, maps, lines, x, 0, max_iter, tol, st);
    if (rc != SENSE_OK) return rc;
  } else {
    int done = 0;
    while (done < max_iter) {
      const int count = (max_iter - done) < kPollEvery ? (max_iter - done) : kPollEvery;
      rc = cg_chunk_graph<St>(pl, maps, lines, x, done, count, tol, st);
      if (rc != SENSE_OK) return rc;
      done += count;
      if (done >= max_iter) break;
      SENSE_CUDA_TRY(cudaMemcpyAsync(pl->live_host, pl->cg(tol).live, sizeof(int), cudaMemcpyDeviceToHost, st));
      SENSE_CUDA_TRY(cudaStreamSynchronize(st));
      if (*pl->live_host <= 0) break;
    }
  }
  rc = plan_centred_output(pl, x, st);
  if (rc != SENSE_OK) return rc;
  PhaseScope ps(pl, SENSE_PHASE_CG_FINISH, st);
  k_cg_finish<<<(sh.frames + 127) / 128, 128, 0, st>>>(pl->cg(tol), sh.frames, iters_out, resid_out, outcome_out, 0);
  return launch_status(cudaGetLastError(), "CG finish");
}

}  // namespace

namespace {

// Sizes and workspace of a plan (allocation only; tables and zeroing follow).
sense_status plan_allocate(sense_plan* pl) {
  const sense_shape& sh = pl->sh;
  const int W = col_width(sh.ny);
  pl->tiles = (sh.nx + W - 1) / W;
  pl->tiles8 = (sh.nx + 7) / 8;
  pl->img = (size_t)sh.ny * sh.nx;
  pl->upd_blocks = (int)((pl->img + UPD_PER_BLOCK - 1) / UPD_PER_BLOCK);
  pl->norm_variant = 0;
  pl->norm_tiles = (sh.nx + normal_variant_width(sh.ny, 0) - 1) / normal_variant_width(sh.ny, 0);
  pl->part_stride = pl->tiles > pl->upd_blocks ? pl->tiles : pl->upd_blocks;
  const int max_tiles = (sh.nx + 3) / 4;  // narrowest tile of any variant
  if (pl->part_stride < max_tiles) pl->part_stride = max_tiles;
  {
    int min_threads = 1 << 30;
    for (int v = 0; v < kNormVariants; ++v) {
      const int th = normal_variant_threads(sh.ny, v);
      if (th > 0 && th < min_threads) min_threads = th;
    }
    pl->max_chunks = update_chunks(pl->img, min_threads);
  }
  const size_t F = (size_t)sh.frames;
  sense_status rc = SENSE_OK;
  if ((pl->own_tw && ((rc = dalloc(pl, &pl->tw_y, (size_t)sh.ny)) != SENSE_OK ||
                      (rc = dalloc(pl, &pl->tw_x, (size_t)sh.nx)) != SENSE_OK)) ||
      (rc = dalloc(pl, &pl->tmp, F * sh.coils * sh.lines * sh.nx)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->r, F * pl->img)) != SENSE_OK || (rc = dalloc(pl, &pl->pp[0], F * pl->img)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->pp[1], F * pl->img)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->q, F * pl->img)) != SENSE_OK || (rc = dalloc(pl, &pl->dbl, 5 * F)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->ints, 3 * F + 2)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->counter, F)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->part, F * pl->part_stride)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->ptable, F)) != SENSE_OK || (rc = dalloc(pl, &pl->pints, 4 * F + 1)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->part_nrm, F * (size_t)max_tiles)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->part_upd, F * (size_t)pl->max_chunks)) != SENSE_OK ||
      (rc = dalloc(pl, &pl->tmap_d, 1)) != SENSE_OK || (rc = dalloc(pl, &pl->fused_ints, F + 1)) != SENSE_OK)
    return rc;
  return SENSE_OK;
}

}  // namespace

namespace sense {

void plan_frames(const sense_plan* pl, const void* S, const int* lines, float2* x, int k0, double tol,
                 PFrame* out, int base) {
  const sense_shape& sh = pl->sh;
  const int F = sh.frames;
  const CgState g = pl->cg(0.0);
  const bool coupled = pl->lambda_t > 0.0;
  for (int f = 0; f < sh.frames; ++f) {
    PFrame& fr = out[f];
    const int sl = coupled ? 0 : f;  // scalar slot: coupled frames share the first frame's
    fr.S = S;
    fr.lines = lines + (size_t)f * sh.lines;
    fr.x = x + (size_t)f * pl->img;
    fr.r = pl->r + (size_t)f * pl->img;
    fr.p[0] = pl->pp[0] + (size_t)f * pl->img;
    fr.p[1] = pl->pp[1] + (size_t)f * pl->img;
    fr.q = pl->q + (size_t)f * pl->img;
    fr.rho = g.rho + sl;
    fr.rho0 = g.rho0 + sl;
    fr.alpha = g.alpha + sl;
    fr.beta = g.beta + sl;
    fr.resid = g.resid + sl;
    fr.iters = g.iters + sl;
    fr.outcome = g.outcome + sl;
    fr.active = g.active + sl;
    fr.coils = sh.coils;
    fr.L = sh.lines;
    fr.tmap = pl->tmap_d;
    fr.k0 = k0;
    fr.kmax = 1 << 30;
    fr.tol = tol;
    fr.lambda = (float)pl->lambda;
    fr.g0 = coupled ? base : base + f;
    fr.gsize = coupled ? F : 1;
    fr.lambda_t = (float)pl->lambda_t;
    fr.nb_prev = base + (f + F - 1) % F;
    fr.nb_next = base + (f + 1) % F;
  }
}

sense_status plan_cg_start(sense_plan* pl, const void* y, const void* S, const int* lines, float2* x, double tol,
                           cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  SENSE_CUDA_TRY(cudaMemsetAsync(pl->counter, 0, sizeof(unsigned) * sh.frames, st));
  SENSE_CUDA_TRY(cudaMemsetAsync(pl->cg(tol).live, 0, sizeof(int), st));
  sense_status rc = sh.storage == SENSE_STORE_BF16 ? run_adjoint<StBF16>(pl, 1, y, S, lines, x, nullptr, tol, st)
                                                   : run_adjoint<StC64>(pl, 1, y, S, lines, x, nullptr, tol, st);
  if (rc != SENSE_OK || pl->lambda_t <= 0.0) return rc;
  k_cg_couple_start<<<1, 32, 0, st>>>(pl->cg(tol), sh.frames);
  return launch_status(cudaGetLastError(), "coupled CG start");
}

std::vector<float2> plan_twiddles(int n) { return twiddles(n); }

sense_status plan_prepare_tmap(sense_plan* pl, const void* S, cudaStream_t st) {
  const sense_shape& sh = pl->sh;
  const int W = normal_variant_width(sh.ny, pl->norm_variant);
  if (pl->tmap_S == S && pl->tmap_W == W) return SENSE_OK;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(SENSE_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const bool bf16 = sh.storage == SENSE_STORE_BF16;
  const cuuint64_t elem = bf16 ? 4 : 8;
  // S viewed as a 2D tensor: [coils * ny] rows of nx elements
  const cuuint64_t dims[2] = {(cuuint64_t)sh.nx, (cuuint64_t)sh.coils * sh.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)sh.nx * elem};
  const cuuint32_t box[2] = {(cuuint32_t)W, (cuuint32_t)(sh.ny <= 256 ? sh.ny : sh.ny / 2)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&pl->tmap_host, bf16 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 2,
                         const_cast<void*>(S), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SENSE_EINVAL, "TMA descriptor of S rejected (code " + std::to_string((int)r) + ")");
  // pageable source: the copy is staged before this call returns
  SENSE_CUDA_TRY(cudaMemcpyAsync(pl->tmap_d, &pl->tmap_host, sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  pl->tmap_S = S;
  pl->tmap_W = W;
  return SENSE_OK;
}

sense_status plan_create_pooled(const sense_shape* shape, int device, cudaStream_t st, const float2* tw_y,
                                const float2* tw_x, sense_plan** out) {
  *out = nullptr;
  sense_status rc = check_shape(shape);
  if (rc != SENSE_OK) return rc;
  sense_plan* pl = new sense_plan();
  pl->sh = *shape;
  pl->device = device;
  pl->pool = st;
  pl->own_tw = false;
  pl->tw_y = const_cast<float2*>(tw_y);
  pl->tw_x = const_cast<float2*>(tw_x);
  if ((rc = plan_allocate(pl)) != SENSE_OK) {
    release(pl);
    delete pl;
    return rc;
  }
  const size_t F = (size_t)pl->sh.frames;
  cudaError_t e = cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->counter, 0, sizeof(unsigned) * F, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->ints, 0, sizeof(int) * (3 * F + 2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->dbl, 0, sizeof(double) * 5 * F, st);
  if (e != cudaSuccess) {
    release(pl);
    delete pl;
    return fail(SENSE_ECUDA, std::string("pooled plan set-up: ") + cudaGetErrorString(e));
  }
  *out = pl;
  return SENSE_OK;
}

void plan_destroy_pooled(sense_plan* pl) {
  if (!pl) return;
  release(pl);
  delete pl;
}

sense_status plan_set_variant_nosync(sense_plan* pl, int variant) {
  const int W = (variant >= 0 && variant < kNormVariants) ? normal_variant_width(pl->sh.ny, variant) : 0;
  if (W <= 0) return fail(SENSE_EINVAL, "no such normal-operator variant");
  pl->norm_variant = variant;
  pl->norm_tiles = (pl->sh.nx + W - 1) / W;
  return SENSE_OK;
}

sense_status plan_cg_finish(sense_plan* pl, int* iters_out, double* resid_out, int* outcome_out, cudaStream_t st) {
  const int F = pl->sh.frames;
  k_cg_finish<<<(F + 127) / 128, 128, 0, st>>>(pl->cg(0.0), F, iters_out, resid_out, outcome_out,
                                                pl->lambda_t > 0.0 ? 1 : 0);
  return launch_status(cudaGetLastError(), "CG finish");
}

}  // namespace sense

extern "C" {

int sense_size_supported(int n) { return size_supported(n) ? 1 : 0; }

const char* sense_last_error(void) { return g_last_error.c_str(); }


sense_status sense_plan_create(const sense_shape* shape, int device, sense_plan** out) {
  sense::TraceRange trace_range("sense_plan_create");
  if (!out) return fail(SENSE_EINVAL, "out is NULL");
  *out = nullptr;
  sense_status rc = check_shape(shape);
  if (rc != SENSE_OK) return rc;
  int ndev = 0;
  SENSE_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(SENSE_EINVAL, "device index out of range");
  DeviceGuard guard(device);
  sense_plan* pl = new sense_plan();
  pl->sh = *shape;
  pl->device = device;
  const sense_shape& sh = pl->sh;
  const size_t F = (size_t)sh.frames;
  if ((rc = plan_allocate(pl)) != SENSE_OK) {
    release(pl);
    delete pl;
    return rc;
  }
  cudaError_t e = cudaMallocHost(&pl->live_host, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&pl->ptable_host, sizeof(PFrame) * F);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->capture_stream, cudaStreamNonBlocking);
  std::vector<float2> ty = twiddles(sh.ny), tx = twiddles(sh.nx);
  if (e == cudaSuccess) e = cudaMemcpy(pl->tw_y, ty.data(), sizeof(float2) * ty.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->tw_x, tx.data(), sizeof(float2) * tx.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(pl->counter, 0, sizeof(unsigned) * F);
  if (e == cudaSuccess) e = cudaMemset(pl->ints, 0, sizeof(int) * (3 * F + 2));
  if (e == cudaSuccess) e = cudaMemset(pl->dbl, 0, sizeof(double) * 5 * F);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    release(pl);
    delete pl;
    return fail(SENSE_ECUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
  }
  *out = pl;
  return SENSE_OK;
}

sense_status sense_plan_destroy(sense_plan* plan) {
  if (!plan) return SENSE_OK;
  DeviceGuard guard(plan->device);
  cudaDeviceSynchronize();
  release(plan);
  delete plan;
  return SENSE_OK;
}

size_t sense_plan_workspace_bytes(const sense_plan* plan) { return plan ? plan->ws_bytes : 0; }

sense_status sense_forward(sense_plan* pl, const sense_c32* x, const void* S, const int32_t* lines, void* y,
                           void* stream) {
  sense::TraceRange trace_range("sense_forward");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(x) || !aligned16(S) || !aligned16(y) || !aligned4(lines))
    return fail(SENSE_EINVAL, "x, S, y must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  DeviceGuard guard(pl->device);
  const float2* xf = reinterpret_cast<const float2*>(x);
  if (pl->sh.storage == SENSE_STORE_BF16) return run_forward<StBF16>(pl, xf, S, lines, y, as_stream(stream));
  return run_forward<StC64>(pl, xf, S, lines, y, as_stream(stream));
}

sense_status sense_adjoint(sense_plan* pl, const void* y, const void* S, const int32_t* lines, sense_c32* x,
                           void* stream) {
  sense::TraceRange trace_range("sense_adjoint");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(x) || !aligned16(S) || !aligned16(y) || !aligned4(lines))
    return fail(SENSE_EINVAL, "x, S, y must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  DeviceGuard guard(pl->device);
  float2* xf = reinterpret_cast<float2*>(x);
  if (pl->sh.storage == SENSE_STORE_BF16)
    return run_adjoint<StBF16>(pl, 0, y, S, lines, xf, nullptr, 0.0, as_stream(stream));
  return run_adjoint<StC64>(pl, 0, y, S, lines, xf, nullptr, 0.0, as_stream(stream));
}

sense_status sense_normal(sense_plan* pl, const sense_c32* x, const void* S, const int32_t* lines, sense_c32* out,
                          void* stream) {
  sense::TraceRange trace_range("sense_normal");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(x) || !aligned16(S) || !aligned16(out) || !aligned4(lines))
    return fail(SENSE_EINVAL, "x, S, out must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  if ((const void*)x == (const void*)out) return fail(SENSE_EINVAL, "out must not alias x");
  DeviceGuard guard(pl->device);
  const float2* xf = reinterpret_cast<const float2*>(x);
  float2* of = reinterpret_cast<float2*>(out);
  if (pl->sh.storage == SENSE_STORE_BF16) return run_normal<StBF16>(pl, xf, S, lines, of, as_stream(stream));
  return run_normal<StC64>(pl, xf, S, lines, of, as_stream(stream));
}

sense_status sense_cg_solve(sense_plan* pl, const void* y, const void* S, const int32_t* lines, int max_iter,
                            double rel_tol, sense_c32* x_out, int32_t* iters_out, double* rel_resid_out,
                            int32_t* outcome_out, void* stream) {
  sense::TraceRange trace_range("sense_cg_solve");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(x_out) || !aligned16(S) || !aligned16(y) || !aligned4(lines))
    return fail(SENSE_EINVAL, "x_out, S, y must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  if (max_iter < 0 || !(rel_tol >= 0.0)) return fail(SENSE_EINVAL, "max_iter must be >= 0 and rel_tol >= 0");
  if ((const void*)x_out == y || (const void*)x_out == S) return fail(SENSE_EINVAL, "x_out aliases an input");
  DeviceGuard guard(pl->device);
  float2* xf = reinterpret_cast<float2*>(x_out);
  if (pl->sh.storage == SENSE_STORE_BF16)
    return run_cg_solve<StBF16>(pl, y, S, lines, max_iter, rel_tol, xf, iters_out, rel_resid_out, outcome_out,
                                as_stream(stream));
  return run_cg_solve<StC64>(pl, y, S, lines, max_iter, rel_tol, xf, iters_out, rel_resid_out, outcome_out,
                             as_stream(stream));
}

sense_status sense_cg_solve_host(sense_plan* pl, const void* y_host, const void* S_host, const int32_t* lines_host,
                                 int max_iter, double rel_tol, sense_c32* x_host, int32_t* iters_host,
                                 double* rel_resid_host, int32_t* outcome_host, void* stream) {
  sense::TraceRange trace_range("sense_cg_solve_host");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!y_host || !S_host || !lines_host || !x_host) return fail(SENSE_EINVAL, "y, S, lines and x must be non-NULL");
  if (max_iter < 0 || !(rel_tol >= 0.0)) return fail(SENSE_EINVAL, "max_iter must be >= 0 and rel_tol >= 0");
  DeviceGuard guard(pl->device);
  const sense_shape& sh = pl->sh;
  const size_t sb = sh.storage == SENSE_STORE_BF16 ? 4 : 8;
  const size_t F = (size_t)sh.frames;
  const size_t y_bytes = F * sh.coils * sh.lines * sh.nx * sb, S_bytes = (size_t)sh.coils * pl->img * sb;
  const size_t l_bytes = F * sh.lines * sizeof(int32_t), x_bytes = F * pl->img * sizeof(float2);
  sense_status rc = SENSE_OK;
  if (!pl->hio_y) {  // first call: device copies of the caller's buffers, owned by the plan
    unsigned char* yb = nullptr;
    unsigned char* sbuf = nullptr;
    if ((rc = dalloc(pl, &yb, y_bytes)) != SENSE_OK || (rc = dalloc(pl, &sbuf, S_bytes)) != SENSE_OK ||
        (rc = dalloc(pl, &pl->hio_lines, F * sh.lines)) != SENSE_OK || (rc = dalloc(pl, &pl->hio_x, F * pl->img)) != SENSE_OK ||
        (rc = dalloc(pl, &pl->hio_ints, 2 * F)) != SENSE_OK || (rc = dalloc(pl, &pl->hio_resid, F)) != SENSE_OK)
      return rc;
    pl->hio_y = yb;
    pl->hio_S = sbuf;
  }
  cudaStream_t st = as_stream(stream);
  SENSE_CUDA_TRY(cudaMemcpyAsync(pl->hio_y, y_host, y_bytes, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(pl->hio_S, S_host, S_bytes, cudaMemcpyHostToDevice, st));
  SENSE_CUDA_TRY(cudaMemcpyAsync(pl->hio_lines, lines_host, l_bytes, cudaMemcpyHostToDevice, st));
  rc = sh.storage == SENSE_STORE_BF16
           ? run_cg_solve<StBF16>(pl, pl->hio_y, pl->hio_S, pl->hio_lines, max_iter, rel_tol, pl->hio_x, pl->hio_ints,
                                  pl->hio_resid, pl->hio_ints + F, st)
           : run_cg_solve<StC64>(pl, pl->hio_y, pl->hio_S, pl->hio_lines, max_iter, rel_tol, pl->hio_x, pl->hio_ints,
                                 pl->hio_resid, pl->hio_ints + F, st);
  if (rc != SENSE_OK) return rc;
  SENSE_CUDA_TRY(cudaMemcpyAsync(x_host, pl->hio_x, x_bytes, cudaMemcpyDeviceToHost, st));
  if (iters_host)
    SENSE_CUDA_TRY(cudaMemcpyAsync(iters_host, pl->hio_ints, F * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (outcome_host)
    SENSE_CUDA_TRY(cudaMemcpyAsync(outcome_host, pl->hio_ints + F, F * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (rel_resid_host)
    SENSE_CUDA_TRY(cudaMemcpyAsync(rel_resid_host, pl->hio_resid, F * sizeof(double), cudaMemcpyDeviceToHost, st));
  return sense_plan_check(pl, stream);  // synchronises `stream`; reports flags the kernels raised
}

sense_status sense_plan_set_column_pass(sense_plan* pl, int staged) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (staged < 0 || staged > 2) return fail(SENSE_EINVAL, "staged must be 0, 1 or 2");
  pl->col_tma = staged;
  return SENSE_OK;
}

sense_status sense_rss(sense_plan* pl, const void* y, const int32_t* lines, float* out, void* stream) {
  sense::TraceRange trace_range("sense_rss");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(y) || !aligned16(out) || !aligned4(lines))
    return fail(SENSE_EINVAL, "y, out must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  DeviceGuard guard(pl->device);
  if (pl->sh.storage == SENSE_STORE_BF16)
    return run_adjoint<StBF16>(pl, 2, y, nullptr, lines, nullptr, out, 0.0, as_stream(stream));
  return run_adjoint<StC64>(pl, 2, y, nullptr, lines, nullptr, out, 0.0, as_stream(stream));
}

sense_status sense_c32_to_bf16(const sense_c32* in, void* out, size_t count, void* stream) {
  if (count == 0) return SENSE_OK;
  if (!aligned4(in) || !aligned4(out)) return fail(SENSE_EINVAL, "in/out must be non-NULL and aligned");
  const unsigned blocks = (unsigned)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
  k_to_bf16<<<blocks, 256, 0, as_stream(stream)>>>(reinterpret_cast<const float2*>(in),
                                                    static_cast<__nv_bfloat162*>(out), count);
  return launch_status(cudaGetLastError(), "bf16 conversion");
}

sense_status sense_plan_set_timing(sense_plan* pl, int on) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  DeviceGuard guard(pl->device);
  collect_spans(pl);
  pl->timing = on ? 1 : 0;
  for (int i = 0; i < SENSE_PHASE_COUNT; ++i) {
    pl->phase_ms[i] = 0.0;
    pl->phase_launches[i] = 0;
  }
  return SENSE_OK;
}

sense_status sense_plan_phase_time(sense_plan* pl, int phase, double* ms_total, long* launches) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (phase < 0 || phase >= SENSE_PHASE_COUNT) return fail(SENSE_EINVAL, "phase out of range");
  DeviceGuard guard(pl->device);
  collect_spans(pl);
  if (ms_total) *ms_total = pl->phase_ms[phase];
  if (launches) *launches = pl->phase_launches[phase];
  return SENSE_OK;
}

sense_status sense_plan_set_cg_mode(sense_plan* pl, int mode) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (mode < 0 || mode > 2) return fail(SENSE_EINVAL, "CG mode must be 0 (graph), 1 (persistent) or 2 (direct)");
  pl->cg_mode = mode;
  return SENSE_OK;
}

sense_status sense_plan_set_variant(sense_plan* pl, int variant) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  const int W = (variant >= 0 && variant < kNormVariants) ? normal_variant_width(pl->sh.ny, variant) : 0;
  if (W <= 0) return fail(SENSE_EINVAL, "no such normal-operator variant for ny=" + std::to_string(pl->sh.ny));
  DeviceGuard guard(pl->device);
  cudaDeviceSynchronize();
  for (auto& kv : pl->graphs) cudaGraphExecDestroy(kv.second);  // graphs bake the old variant in
  pl->graphs.clear();
  pl->norm_variant = variant;
  pl->norm_tiles = (pl->sh.nx + W - 1) / W;
  return SENSE_OK;
}

int sense_plan_variant(const sense_plan* pl) { return pl ? pl->norm_variant : -1; }

sense_status sense_plan_set_temporal(sense_plan* pl, double lambda_t) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!(lambda_t >= 0.0) || !std::isfinite(lambda_t) || lambda_t > 3.0e38)
    return fail(SENSE_EINVAL, "lambda_t must be finite, >= 0 and representable in FP32");
  if (lambda_t == pl->lambda_t) return SENSE_OK;
  DeviceGuard guard(pl->device);
  cudaDeviceSynchronize();
  pl->ptable_key[0] = nullptr;  // the persistent frame table bakes the coupling in
  pl->lambda_t = lambda_t;
  return SENSE_OK;
}

sense_status sense_plan_set_lambda(sense_plan* pl, double lambda) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!(lambda >= 0.0) || !std::isfinite(lambda) || lambda > 3.0e38)
    return fail(SENSE_EINVAL, "lambda must be finite, >= 0 and representable in FP32");
  if (lambda == pl->lambda) return SENSE_OK;
  DeviceGuard guard(pl->device);
  cudaDeviceSynchronize();
  for (auto& kv : pl->graphs) cudaGraphExecDestroy(kv.second);  // graphs bake lambda in
  pl->graphs.clear();
  pl->ptable_key[0] = nullptr;  // and so does the persistent frame table
  pl->lambda = lambda;
  return SENSE_OK;
}

sense_status sense_plan_autotune(sense_plan* pl, const void* S, const int32_t* lines, int* variant_out,
                                 double* ms_out, void* stream) {
  sense::TraceRange trace_range("sense_plan_autotune");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (!aligned16(S) || !aligned4(lines)) return fail(SENSE_EINVAL, "S must be 16-byte aligned, lines 4-byte");
  DeviceGuard guard(pl->device);
  const sense_shape& sh = pl->sh;
  const bool persistent = pl->cg_mode == 1;
  const TuneKey key{pl->device, sh.ny, sh.nx, sh.coils, sh.frames, sh.lines, sh.storage, persistent ? 1 : 0};
  int best = tune_cache_lookup(key);
  if (ms_out)
    for (int v = 0; v < kNormVariants; ++v) ms_out[v] = -1.0;
  cudaStream_t st = as_stream(stream);
  if (best < 0) {
    // Persistent mode times a short fixed-length CG solve, whose cost the
    // kernel variant decides together with the block count per SM; the
    // right-hand side is a constant k-space pattern on the sampled lines, so
    // no frame breaks down early.  Otherwise one normal-operator launch.
    const bool bf16 = sh.storage == SENSE_STORE_BF16;
    const size_t y_bytes = (size_t)sh.frames * sh.coils * sh.lines * sh.nx * (bf16 ? 4 : 8);
    void* y_tmp = nullptr;
    float2* x_tmp = nullptr;
    if (persistent) {
      SENSE_CUDA_TRY(cudaStreamSynchronize(st));
      SENSE_CUDA_TRY(cudaMalloc(&y_tmp, y_bytes));
      if (cudaMalloc(&x_tmp, sizeof(float2) * pl->img * sh.frames) != cudaSuccess) {
        cudaFree(y_tmp);
        return fail(SENSE_ENOMEM, "autotune scratch");
      }
      cudaMemsetAsync(y_tmp, 0x3c, y_bytes, st);  // every component 0x3c3c.. > 0
    } else {
      SENSE_CUDA_TRY(cudaMemsetAsync(pl->r, 0, sizeof(float2) * pl->img * sh.frames, st));
    }
    constexpr int kTuneIters = 10;
    auto run_once = [&]() -> sense_status {
      if (persistent)
        return bf16 ? run_cg_solve<StBF16>(pl, y_tmp, S, lines, kTuneIters, 0.0, x_tmp, nullptr, nullptr, nullptr, st)
                    : run_cg_solve<StC64>(pl, y_tmp, S, lines, kTuneIters, 0.0, x_tmp, nullptr, nullptr, nullptr, st);
      return bf16 ? run_normal<StBF16>(pl, pl->r, S, lines, pl->q, st)
                  : run_normal<StC64>(pl, pl->r, S, lines, pl->q, st);
    };
    cudaEvent_t a = nullptr, b = nullptr;
    sense_status rc = SENSE_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
      rc = fail(SENSE_ECUDA, "autotune events");
    double best_ms = 1e30;
    const int warm = persistent ? 1 : 3, reps = persistent ? 3 : 10;
    const int saved_timing = pl->timing;
    pl->timing = 0;
    for (int v = 0; v < kNormVariants && rc == SENSE_OK; ++v) {
      if (normal_variant_width(sh.ny, v) <= 0) continue;
      rc = sense_plan_set_variant(pl, v);
      for (int it = 0; it < warm && rc == SENSE_OK; ++it) rc = run_once();
      if (rc != SENSE_OK) break;
      cudaEventRecord(a, st);
      for (int it = 0; it < reps && rc == SENSE_OK; ++it) rc = run_once();
      cudaEventRecord(b, st);
      if (rc != SENSE_OK) break;
      float ms = 0.f;
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      const double per = ms / reps;
      if (ms_out) ms_out[v] = per;
      if (per < best_ms) {
        best_ms = per;
        best = v;
      }
    }
    pl->timing = saved_timing;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (persistent) {
      cudaStreamSynchronize(st);
      cudaFree(y_tmp);
      cudaFree(x_tmp);
    }
    if (rc == SENSE_OK) rc = sense_plan_check(pl, stream);
    if (rc != SENSE_OK) return rc;
    if (best < 0) return fail(SENSE_ECUDA, "autotune found no runnable variant");
    tune_cache_store(key, best);
  }
  sense_status rc = sense_plan_set_variant(pl, best);
  if (rc != SENSE_OK) return rc;
  if (variant_out) *variant_out = best;
  return SENSE_OK;
}

sense_status sense_selftest_wait(int device, long max_spins) {
  if (max_spins < 1 || max_spins > (1L << 20)) return fail(SENSE_EINVAL, "max_spins must be in [1, 2^20]");
  int ndev = 0;
  SENSE_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(SENSE_EINVAL, "device index out of range");
  DeviceGuard guard(device);
  int* d = nullptr;  // [0] the flag nobody sets, [1] the result
  SENSE_CUDA_TRY(cudaMalloc(&d, 2 * sizeof(int)));
  int res[2] = {0, -1};
  cudaError_t e = cudaMemcpy(d, res, sizeof(res), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>(d, max_spins, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(res, d, sizeof(res), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(SENSE_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  if (res[1] == 1) return fail(SENSE_ETIMEOUT, "the bounded wait gave up as designed");
  return fail(SENSE_ECUDA, "the bounded wait returned without timing out");
}

sense_status sense_plan_check(sense_plan* pl, void* stream) {
  sense::TraceRange trace_range("sense_plan_check");
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  DeviceGuard guard(pl->device);
  SENSE_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
  int flags = 0;
  SENSE_CUDA_TRY(cudaMemcpy(&flags, pl->err(), sizeof(int), cudaMemcpyDeviceToHost));
  SENSE_CUDA_TRY(cudaMemset(pl->err(), 0, sizeof(int)));
  if (flags & ERR_LINES)
    return fail(SENSE_EDEVICE, "a line index was outside [0, ny) or lines were not strictly increasing");
  if (flags & ERR_TIMEOUT) return fail(SENSE_ETIMEOUT, "a bounded device-side wait gave up");
  return SENSE_OK;
}

}  // extern "C"

extern "C" void sense_testing_staggered_item(long long t, int units, int first_items, int second_items, int lag,
                                             int out[3]) {
  const sense::StaggeredItem it = sense::staggered_item((long)t, units, first_items, second_items, lag);
  out[0] = it.second;
  out[1] = it.unit;
  out[2] = it.piece;
}

extern "C" int sense_testing_persistent_lag(int frames, int tiles, int grid) {
  return sense::persistent_lag(frames, tiles, grid);
}

extern "C" sense_status sense_testing_plan_set_order(sense_plan* pl, int order) {
  if (!pl) return fail(SENSE_EINVAL, "plan is NULL");
  if (order < sense::kOrderAuto) return fail(SENSE_EINVAL, "order must be -1, -2 or a lag >= 0");
  pl->cg_order = order;
  return SENSE_OK;
}
