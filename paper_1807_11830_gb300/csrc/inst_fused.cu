// Launchers of the single-launch fused operators (fused.cuh): square images
// whose length has a TMA column pass.
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "fused.cuh"
#include "launch.h"

namespace sense {

namespace {

constexpr int kFusedMaxSmem = 227 * 1024;

// One wave of resident blocks (the schedule's waits need every ticket holder running).
template <class K>
cudaError_t fused_grid(K kern, int threads, size_t smem, long items, int sms, int* grid) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> occ_cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ_cache.find({dev, smem});
    if (it != occ_cache.end()) occ = it->second;
  }
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorNotSupported;
    std::lock_guard<std::mutex> lk(mu);
    occ_cache[{dev, smem}] = occ;
  }
  const long cap = (long)sms * occ;
  *grid = (int)(items < cap ? items : cap);
  return cudaSuccess;
}

template <int N, class St, class YSt, int MODE>
cudaError_t adj_fused_n(const CUtensorMap& tmK, const CUtensorMap& tmS, const AdjColArgs<St>& a, const void* y,
                        float2* tmp_out, const FusedSched& sc, float cs, int sms, cudaStream_t s) {
  static unsigned long long done = 0;
  const size_t smem = fused_smem_bytes<N, St>(a.L, true);
  if (smem > (size_t)kFusedMaxSmem) return cudaErrorNotSupported;
  // the kernel also holds a few words of static shared memory: the dynamic limit is the largest any L needs
  cudaError_t e = ensure_smem(k_adjoint_fused<N, St, YSt, MODE>, fused_smem_bytes<N, St>(N, true), &done);
  const long items = (long)sc.frames * (sc.first_tiles + sc.second_tiles);
  if (e != cudaSuccess || items == 0) return e;
  int grid = 0;
  e = fused_grid(k_adjoint_fused<N, St, YSt, MODE>, ColTma<N>::C::THREADS, smem, items, sms, &grid);
  if (e != cudaSuccess) return e;
  k_adjoint_fused<N, St, YSt, MODE><<<grid, ColTma<N>::C::THREADS, smem, s>>>(
      tmK, tmS, a, static_cast<const typename YSt::T*>(y), tmp_out, sc, cs);
  return cudaGetLastError();
}

template <int N, class St>
cudaError_t fwd_fused_n(const CUtensorMap& tmS, const FwdColArgs<St>& a, void* y, const FusedSched& sc, float cs,
                        int sms, cudaStream_t s) {
  static unsigned long long done = 0;
  const size_t smem = fused_smem_bytes<N, St>(a.L, false);
  if (smem > (size_t)kFusedMaxSmem) return cudaErrorNotSupported;
  cudaError_t e = ensure_smem(k_forward_fused<N, St>, fused_smem_bytes<N, St>(N, false), &done);
  const long items = (long)sc.frames * (sc.first_tiles + sc.second_tiles);
  if (e != cudaSuccess || items == 0) return e;
  int grid = 0;
  e = fused_grid(k_forward_fused<N, St>, ColTma<N>::C::THREADS, smem, items, sms, &grid);
  if (e != cudaSuccess) return e;
  k_forward_fused<N, St><<<grid, ColTma<N>::C::THREADS, smem, s>>>(tmS, a, static_cast<typename St::T*>(y), sc, cs);
  return cudaGetLastError();
}

#define SENSE_FOR_EACH_FUSED_SIZE(X) X(64) X(96) X(120) X(128) X(144) X(160) X(192) X(240) X(256) X(288) X(320) X(384)

}  // namespace

template <class St>
cudaError_t launch_adjoint_fused(int n, int mode, bool y_bf16, const CUtensorMap& tmK, const CUtensorMap& tmS,
                                 const AdjColArgs<St>& a, const void* y, float2* tmp_out, const FusedSched& sc,
                                 float cs, int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N)                                                                                     \
  case N:                                                                                                 \
    if constexpr (ColTma<N>::ok) {                                                                        \
      if (mode == 0) return adj_fused_n<N, St, St, 0>(tmK, tmS, a, y, tmp_out, sc, cs, sms, s);           \
      if (mode == 1) return adj_fused_n<N, St, St, 1>(tmK, tmS, a, y, tmp_out, sc, cs, sms, s);           \
      if constexpr (std::is_same<St, StC64>::value) {                                                     \
        if (mode == 2 && y_bf16) return adj_fused_n<N, StC64, StBF16, 2>(tmK, tmS, a, y, tmp_out, sc, cs, sms, s); \
        if (mode == 2) return adj_fused_n<N, StC64, StC64, 2>(tmK, tmS, a, y, tmp_out, sc, cs, sms, s);   \
      }                                                                                                   \
    }                                                                                                     \
    return cudaErrorNotSupported;
    SENSE_FOR_EACH_FUSED_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorNotSupported;
  }
}

template <class St>
cudaError_t launch_forward_fused(int n, const CUtensorMap& tmS, const FwdColArgs<St>& a, void* y, const FusedSched& sc,
                                 float cs, int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N)                                                                       \
  case N:                                                                                   \
    if constexpr (ColTma<N>::ok) return fwd_fused_n<N, St>(tmS, a, y, sc, cs, sms, s);      \
    return cudaErrorNotSupported;
    SENSE_FOR_EACH_FUSED_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorNotSupported;
  }
}

template cudaError_t launch_adjoint_fused<StC64>(int, int, bool, const CUtensorMap&, const CUtensorMap&,
                                                 const AdjColArgs<StC64>&, const void*, float2*, const FusedSched&,
                                                 float, int, cudaStream_t);
template cudaError_t launch_adjoint_fused<StBF16>(int, int, bool, const CUtensorMap&, const CUtensorMap&,
                                                  const AdjColArgs<StBF16>&, const void*, float2*, const FusedSched&,
                                                  float, int, cudaStream_t);
template cudaError_t launch_forward_fused<StC64>(int, const CUtensorMap&, const FwdColArgs<StC64>&, void*,
                                                 const FusedSched&, float, int, cudaStream_t);
template cudaError_t launch_forward_fused<StBF16>(int, const CUtensorMap&, const FwdColArgs<StBF16>&, void*,
                                                  const FusedSched&, float, int, cudaStream_t);

}  // namespace sense
