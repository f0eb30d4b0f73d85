// Launchers of the TMA-staged persistent column passes (colpass.cuh), both
// storages of S.  Lengths from 64 up whose 8-column tile fills whole warps
// have them; the others keep the register-staged column kernels.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <utility>

#include "colpass.cuh"
#include "launch.h"

namespace sense {

namespace {

constexpr int kMaxDynSmem = 227 * 1024;

// One wave of resident blocks (at most one block per item).  The occupancy
// query is remembered per (kernel, device, shared-memory size).
template <class K>
cudaError_t coltma_grid(K kern, int threads, size_t smem, long items, int sms, int* grid) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> occ_cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(reinterpret_cast<const void*>(kern), dev, smem);
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ_cache.find(key);
    if (it != occ_cache.end()) occ = it->second;
  }
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorNotSupported;
    std::lock_guard<std::mutex> lk(mu);
    occ_cache[key] = occ;
  }
  const long cap = (long)sms * occ;
  *grid = (int)(items < cap ? items : cap);
  return cudaSuccess;
}

template <int N, class St, int MODE>
cudaError_t adj_tma_n(const CUtensorMap& tmK, const CUtensorMap& tmS, const AdjColArgs<St>& a, int frames, int sms,
                      cudaStream_t s) {
  static unsigned long long done = 0;
  const size_t smem = coltma_smem_bytes<N, St>(a.L, true);
  if (smem > (size_t)kMaxDynSmem) return cudaErrorNotSupported;
  cudaError_t e = ensure_smem(k_adj_col_tma<N, St, MODE>, kMaxDynSmem, &done);
  const long items = (long)a.tiles * frames;
  if (e != cudaSuccess || items == 0) return e;
  int grid = 0;
  e = coltma_grid(k_adj_col_tma<N, St, MODE>, ColTma<N>::C::THREADS, smem, items, sms, &grid);
  if (e != cudaSuccess) return e;
  k_adj_col_tma<N, St, MODE><<<grid, ColTma<N>::C::THREADS, smem, s>>>(tmK, tmS, a, frames);
  return cudaGetLastError();
}

template <int N, class St>
cudaError_t fwd_tma_n(const CUtensorMap& tmS, const FwdColArgs<St>& a, int tiles, int frames, int sms,
                      cudaStream_t s) {
  static unsigned long long done = 0;
  const size_t smem = coltma_smem_bytes<N, St>(a.L, false);
  if (smem > (size_t)kMaxDynSmem) return cudaErrorNotSupported;
  cudaError_t e = ensure_smem(k_fwd_col_tma<N, St>, kMaxDynSmem, &done);
  const long items = (long)tiles * frames;
  if (e != cudaSuccess || items == 0) return e;
  int grid = 0;
  e = coltma_grid(k_fwd_col_tma<N, St>, ColTma<N>::C::THREADS, smem, items, sms, &grid);
  if (e != cudaSuccess) return e;
  k_fwd_col_tma<N, St><<<grid, ColTma<N>::C::THREADS, smem, s>>>(tmS, a, tiles, frames);
  return cudaGetLastError();
}

#define SENSE_FOR_EACH_TMA_SIZE(X) X(64) X(96) X(120) X(128) X(144) X(160) X(192) X(240) X(256) X(288) X(320) X(384)

}  // namespace

bool coltma_supported(int n) {
  switch (n) {
#define SENSE_CASE(N) case N: return ColTma<N>::ok;
    SENSE_FOR_EACH_TMA_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return false;
  }
}

template <class St>
cudaError_t launch_adj_col_tma(int n, int mode, const CUtensorMap& tmK, const CUtensorMap& tmS,
                               const AdjColArgs<St>& a, int frames, int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N)                                                                          \
  case N:                                                                                      \
    if constexpr (ColTma<N>::ok) {                                                             \
      if (mode == 0) return adj_tma_n<N, St, 0>(tmK, tmS, a, frames, sms, s);                  \
      if (mode == 1) return adj_tma_n<N, St, 1>(tmK, tmS, a, frames, sms, s);                  \
      if constexpr (std::is_same<St, StC64>::value)                                            \
        if (mode == 2) return adj_tma_n<N, St, 2>(tmK, tmS, a, frames, sms, s);                \
    }                                                                                          \
    return cudaErrorNotSupported;
    SENSE_FOR_EACH_TMA_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorNotSupported;
  }
}

template <class St>
cudaError_t launch_fwd_col_tma(int n, const CUtensorMap& tmS, const FwdColArgs<St>& a, int tiles, int frames,
                               int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N)                                                    \
  case N:                                                                \
    if constexpr (ColTma<N>::ok) return fwd_tma_n<N, St>(tmS, a, tiles, frames, sms, s); \
    return cudaErrorNotSupported;
    SENSE_FOR_EACH_TMA_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorNotSupported;
  }
}

template cudaError_t launch_adj_col_tma<StC64>(int, int, const CUtensorMap&, const CUtensorMap&,
                                               const AdjColArgs<StC64>&, int, int, cudaStream_t);
template cudaError_t launch_adj_col_tma<StBF16>(int, int, const CUtensorMap&, const CUtensorMap&,
                                                const AdjColArgs<StBF16>&, int, int, cudaStream_t);
template cudaError_t launch_fwd_col_tma<StC64>(int, const CUtensorMap&, const FwdColArgs<StC64>&, int, int, int,
                                               cudaStream_t);
template cudaError_t launch_fwd_col_tma<StBF16>(int, const CUtensorMap&, const FwdColArgs<StBF16>&, int, int, int,
                                                cudaStream_t);

}  // namespace sense
