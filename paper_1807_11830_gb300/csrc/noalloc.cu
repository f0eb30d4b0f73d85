// Allocation-free variant of the adjoint E^H (sense_adjoint_noalloc).
//
// Some callers cannot allocate device memory: plugins running inside a host
// application that owns all device memory through its own pool allocator,
// processes whose device memory budget is fixed before they start, and
// latency-critical loops that must not enter the CUDA allocator (cudaMalloc
// and cudaFree can synchronise the device).  They cannot create a plan,
// because a plan allocates its workspace.  This entry point needs no plan: the
// intermediate between the row and column passes lives in a file-scope
// __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.  Twiddle tables for every supported length and the
// kernels' error word live in file-scope arrays too.
//
// Device-side addresses of those arrays are taken once per device with
// cudaGetSymbolAddress while that device is current; the host-side names of
// the arrays are stand-ins and are never passed to a kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"
#include "trace.h"
#include "sense.h"

using namespace sense;

namespace sense {
// Stores the message sense_last_error() returns on this thread (sense_api.cu).
void record_error(const std::string& msg);
}  // namespace sense

namespace {

// Largest intermediate, in complex values: frames * coils * lines * nx.
constexpr size_t kScratchComplex = size_t(1) << 21;  // 16 MiB
// Twiddles of every supported length, back to back in SENSE_FOR_EACH_SIZE order.
#define SENSE_PLUS(N) +N
constexpr int kTwiddleTotal = 0 SENSE_FOR_EACH_SIZE(SENSE_PLUS);
#undef SENSE_PLUS
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_scratch[kScratchComplex];
static __device__ __align__(256) float2 g_twiddles[kTwiddleTotal];
static __device__ __align__(256) int g_err[4];

struct DeviceTables {
  bool ready = false;
  float2* scratch = nullptr;
  float2* twiddles = nullptr;
  int* err = nullptr;
};

std::mutex g_setup_mutex;
DeviceTables g_tables[kMaxDevices];

int twiddle_offset(int n) {
  int off = 0;
#define SENSE_OFF(N)      \
  if (n == N) return off; \
  off += N;
  SENSE_FOR_EACH_SIZE(SENSE_OFF)
#undef SENSE_OFF
  return -1;
}

// Set-up of the current device: device addresses of the file-scope arrays,
// and the twiddle tables (FP64 angles rounded once to FP32, the same values a
// plan uploads).  Runs once per device under a mutex.
sense_status setup_current_device(int dev, DeviceTables** out, std::string* msg) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceTables& t = g_tables[dev];
  if (!t.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      *msg = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
      return SENSE_ECUDA;
    }
    t.scratch = static_cast<float2*>(p);
    e = cudaGetSymbolAddress(&p, g_twiddles);
    if (e != cudaSuccess) {
      *msg = std::string("cudaGetSymbolAddress(twiddles): ") + cudaGetErrorString(e);
      return SENSE_ECUDA;
    }
    t.twiddles = static_cast<float2*>(p);
    e = cudaGetSymbolAddress(&p, g_err);
    if (e != cudaSuccess) {
      *msg = std::string("cudaGetSymbolAddress(err): ") + cudaGetErrorString(e);
      return SENSE_ECUDA;
    }
    t.err = static_cast<int*>(p);
    std::vector<float2> host((size_t)kTwiddleTotal);
    const double two_pi = 6.283185307179586476925286766559;
    size_t k = 0;
#define SENSE_TW(N)                                                     \
  for (int m = 0; m < N; ++m, ++k) {                                    \
    const double a = -two_pi * (double)m / (double)N;                   \
    host[k] = make_float2((float)std::cos(a), (float)std::sin(a));      \
  }
    SENSE_FOR_EACH_SIZE(SENSE_TW)
#undef SENSE_TW
    e = cudaMemcpyToSymbol(g_twiddles, host.data(), sizeof(float2) * host.size());
    if (e != cudaSuccess) {
      *msg = std::string("twiddle upload: ") + cudaGetErrorString(e);
      return SENSE_ECUDA;
    }
    t.ready = true;
  }
  *out = &t;
  return SENSE_OK;
}

template <class St>
sense_status noalloc_adjoint(const sense_shape& sh, const DeviceTables& t, const void* y, const void* S,
                             const int32_t* lines, float2* x, cudaStream_t st, std::string* msg) {
  RowArgs<typename St::T, float2> ra{};
  ra.in = static_cast<const typename St::T*>(y);
  ra.out = t.scratch;
  ra.tw = t.twiddles + twiddle_offset(sh.nx);
  ra.rows = (long)sh.frames * sh.coils * sh.lines;
  ra.centred = sh.centred;
  ra.cs = ((sh.ny / 2 + sh.nx / 2) & 1) ? -1.0f : 1.0f;
  ra.err = t.err;
  cudaError_t e = launch_rows_inv<St>(sh.nx, ra, st);
  if (e != cudaSuccess) {
    *msg = std::string("adjoint row pass: ") + cudaGetErrorString(e);
    return SENSE_ECUDA;
  }
  const int W = col_width(sh.ny);
  const int tiles = (sh.nx + W - 1) / W;
  AdjColArgs<St> a{};
  a.tmp = t.scratch;
  a.S = static_cast<const typename St::T*>(S);
  a.lines = lines;
  a.tw = t.twiddles + twiddle_offset(sh.ny);
  a.x = x;
  a.nx = sh.nx;
  a.coils = sh.coils;
  a.L = sh.lines;
  a.tiles = tiles;
  a.centred = sh.centred;
  a.err = t.err;
  e = launch_adj_col<St>(sh.ny, 0, a, tiles, sh.frames, st);
  if (e != cudaSuccess) {
    *msg = std::string("adjoint column pass: ") + cudaGetErrorString(e);
    return SENSE_ECUDA;
  }
  return SENSE_OK;
}

}  // namespace

extern "C" sense_status sense_adjoint_noalloc(const sense_shape* shape, const void* y, const void* S,
                                              const int32_t* lines, sense_c32* x, void* stream) {
  sense::TraceRange trace_range("sense_adjoint_noalloc");
  sense_status rc = SENSE_OK;
  std::string msg;
  auto done = [&](sense_status s, const std::string& m) {
    if (s != SENSE_OK) sense::record_error(m);
    return s;
  };
  if (!shape) return done(SENSE_EINVAL, "shape is NULL");
  const sense_shape& sh = *shape;
  if (sh.frames < 1 || sh.coils < 1 || sh.lines < 1 || sh.lines > sh.ny || sh.frames > 65535)
    return done(SENSE_EINVAL, "need frames in [1, 65535], coils >= 1, lines in [1, ny]");
  if (sh.storage != SENSE_STORE_C64 && sh.storage != SENSE_STORE_BF16)
    return done(SENSE_EINVAL, "storage must be SENSE_STORE_C64 or SENSE_STORE_BF16");
  if (sh.centred != 0 && sh.centred != 1) return done(SENSE_EINVAL, "centred must be 0 or 1");
  if (!size_supported(sh.ny) || !size_supported(sh.nx))
    return done(SENSE_EUNSUPPORTED_SIZE, "no compiled transform for this ny / nx");
  const size_t need = (size_t)sh.frames * sh.coils * sh.lines * sh.nx;
  if (need > kScratchComplex)
    return done(SENSE_EINVAL, "frames*coils*lines*nx = " + std::to_string(need) +
                                  " exceeds the allocation-free scratch of " + std::to_string(kScratchComplex) +
                                  " complex values; use sense_adjoint with a plan");
  auto a16 = [](const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!a16(y) || !a16(S) || !a16(x) || lines == nullptr || (reinterpret_cast<uintptr_t>(lines) & 3u))
    return done(SENSE_EINVAL, "y, S, x must be non-NULL and 16-byte aligned; lines 4-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return done(SENSE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return done(SENSE_EINVAL, "device index beyond the supported range");
  DeviceTables* t = nullptr;
  rc = setup_current_device(dev, &t, &msg);
  if (rc != SENSE_OK) return done(rc, msg);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float2* xf = reinterpret_cast<float2*>(x);
  if (sh.storage == SENSE_STORE_BF16)
    rc = noalloc_adjoint<StBF16>(sh, *t, y, S, lines, xf, st, &msg);
  else
    rc = noalloc_adjoint<StC64>(sh, *t, y, S, lines, xf, st, &msg);
  return done(rc, msg);
}

