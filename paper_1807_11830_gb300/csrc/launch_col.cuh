// Launcher templates of the column and row kernels (included by the
// per-family instantiation units so the families compile in parallel).
#pragma once
#include "launch.h"
#include "persistent.cuh"

namespace sense {

template <int N, class St>
cudaError_t fwd_col_n(const FwdColArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = col_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_fwd_col<N, St>, sm, &done);
  if (e != cudaSuccess || tiles == 0 || frames == 0) return e;
  k_fwd_col<N, St><<<dim3(tiles, frames), ColPass<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, class St, int MODE>
cudaError_t adj_col_n(const AdjColArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = col_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_adj_col<N, St, MODE>, sm, &done);
  if (e != cudaSuccess || tiles == 0 || frames == 0) return e;
  k_adj_col<N, St, MODE><<<dim3(tiles, frames), ColPass<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, int V, class St, bool CG>
cudaError_t normal_nv(const NormalArgs<St>& a, int frames, cudaStream_t s) {
  if constexpr (!NormCfg<N, V>::exists) {
    return cudaErrorInvalidValue;
  } else {
    using C = typename NormCfg<N, V>::C;
    static unsigned long long done = 0;
    constexpr size_t sm = normal_smem_bytes<C, St>();
    static_assert(sm <= 227 * 1024, "normal kernel shared memory");
    cudaError_t e = ensure_smem(k_normal<N, V, St, CG>, sm, &done);
    const int tiles = (a.nx + C::W - 1) / C::W;
    if (e != cudaSuccess || frames == 0) return e;  // no frames: attribute set-up only
    k_normal<N, V, St, CG><<<dim3(tiles, frames), C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
  }
}

template <int N, class St, bool CG>
cudaError_t normal_n(int variant, const NormalArgs<St>& a, int frames, cudaStream_t s) {
  switch (variant) {
    case 0: return normal_nv<N, 0, St, CG>(a, frames, s);
    case 1: return normal_nv<N, 1, St, CG>(a, frames, s);
    case 2: return normal_nv<N, 2, St, CG>(a, frames, s);
    case 3: return normal_nv<N, 3, St, CG>(a, frames, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int V, class St>
cudaError_t persistent_nv(const PArgs& a, int sms, cudaStream_t s) {
  if constexpr (!NormCfg<N, V>::exists) {
    return cudaErrorInvalidValue;
  } else {
    using C = typename NormCfg<N, V>::C;
    static unsigned long long done = 0;
    constexpr size_t sm = persistent_smem_bytes<C, St>();
    static_assert(sm <= 227 * 1024, "persistent kernel shared memory");
    cudaError_t e = ensure_smem(k_cg_persistent<N, V, St>, sm, &done);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persistent<N, V, St>, C::THREADS, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (a.nframes == 0 || a.iters == 0) return cudaSuccess;  // attribute set-up only
    PArgs b = a;
    if (b.lag == kOrderAuto) b.lag = persistent_lag(b.nframes, b.tiles, sms * per_sm);
    if (b.lag < kOrderIterationMajor || (b.lag > 0 && b.lag >= b.nframes)) return cudaErrorInvalidValue;  // D < frames
    k_cg_persistent<N, V, St><<<sms * per_sm, C::THREADS, sm, s>>>(b);
    return cudaGetLastError();
  }
}

template <int N, int V, class St>
int persistent_resident_nv() {
  if constexpr (!NormCfg<N, V>::exists) {
    return 0;
  } else {
    using C = typename NormCfg<N, V>::C;
    static unsigned long long done = 0;
    constexpr size_t sm = persistent_smem_bytes<C, St>();
    if (ensure_smem(k_cg_persistent<N, V, St>, sm, &done) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persistent<N, V, St>, C::THREADS, sm) !=
        cudaSuccess)
      return 0;
    return per_sm;
  }
}

template <int N, class St>
int persistent_resident_n(int variant) {
  switch (variant) {
    case 0: return persistent_resident_nv<N, 0, St>();
    case 1: return persistent_resident_nv<N, 1, St>();
    case 2: return persistent_resident_nv<N, 2, St>();
    case 3: return persistent_resident_nv<N, 3, St>();
    default: return 0;
  }
}

template <int N, class St>
cudaError_t persistent_n(int variant, const PArgs& a, int sms, cudaStream_t s) {
  switch (variant) {
    case 0: return persistent_nv<N, 0, St>(a, sms, s);
    case 1: return persistent_nv<N, 1, St>(a, sms, s);
    case 2: return persistent_nv<N, 2, St>(a, sms, s);
    case 3: return persistent_nv<N, 3, St>(a, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
constexpr int norm_variant_threads(int v) {
  return v == 0 ? NormCfg<N, 0>::C::THREADS
       : v == 1 ? (NormCfg<N, 1>::exists ? NormCfg<N, 1>::C::THREADS : 0)
       : v == 2 ? (NormCfg<N, 2>::exists ? NormCfg<N, 2>::C::THREADS : 0)
       : v == 3 ? (NormCfg<N, 3>::exists ? NormCfg<N, 3>::C::THREADS : 0) : 0;
}

template <int N>
constexpr int norm_variant_width(int v) {
  return v == 0 ? NormCfg<N, 0>::C::W
       : v == 1 ? (NormCfg<N, 1>::exists ? NormCfg<N, 1>::C::W : 0)
       : v == 2 ? (NormCfg<N, 2>::exists ? NormCfg<N, 2>::C::W : 0)
       : v == 3 ? (NormCfg<N, 3>::exists ? NormCfg<N, 3>::C::W : 0) : 0;
}

// 1 if the variant's normal-operator tiles read the transposed maps S^T
template <int N>
constexpr int norm_variant_transposed(int v) {
  return v == 0 ? (int)is_wcol<typename NormCfg<N, 0>::C>::value
       : v == 1 ? (NormCfg<N, 1>::exists ? (int)is_wcol<typename NormCfg<N, 1>::C>::value : 0)
       : v == 2 ? (NormCfg<N, 2>::exists ? (int)is_wcol<typename NormCfg<N, 2>::C>::value : 0)
       : v == 3 ? (NormCfg<N, 3>::exists ? (int)is_wcol<typename NormCfg<N, 3>::C>::value : 0) : 0;
}

// Complex64 in and out with 16-byte aligned pointers: the persistent
// bulk-copy row kernel, one wave of resident blocks.
template <int N, int DIR>
cudaError_t rows_bulk_n(const RowArgs<float2, float2>& a, cudaStream_t s) {
  static unsigned long long done = 0;
  static int resident[64] = {0};  // blocks per SM, per device
  constexpr size_t sm = row_bulk_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_rows_bulk<N, DIR>, sm, &done);
  if (e != cudaSuccess) return e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  int& per_sm = resident[dev & 63];
  if (per_sm == 0) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_bulk<N, DIR>, RowPass<N>::C::THREADS, sm);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long tiles = (a.rows + RowPass<N>::C::W - 1) / RowPass<N>::C::W;
  if (tiles <= 0) return cudaSuccess;
  const long grid = tiles < (long)sms * per_sm ? tiles : (long)sms * per_sm;
  k_rows_bulk<N, DIR><<<(unsigned)grid, RowPass<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR, class InSt, class OutSt>
cudaError_t rows_n(const RowArgs<typename InSt::T, typename OutSt::T>& a, cudaStream_t s) {
  if constexpr (std::is_same<typename InSt::T, float2>::value && std::is_same<typename OutSt::T, float2>::value &&
                RowPass<N>::P == N + 2) {
    if (a.rows <= 0) {  // attribute set-up only (before a graph capture): both kernels
      const cudaError_t e = rows_bulk_n<N, DIR>(a, s);
      if (e != cudaSuccess) return e;
    } else if ((reinterpret_cast<uintptr_t>(a.in) & 15u) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0) {
      return rows_bulk_n<N, DIR>(a, s);
    }
  }
  static unsigned long long done = 0;
  constexpr size_t sm = row_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_rows<N, DIR, InSt, OutSt>, sm, &done);
  if (e != cudaSuccess) return e;
  const long blocks = (a.rows + RowPass<N>::C::W - 1) / RowPass<N>::C::W;
  if (blocks <= 0) return cudaSuccess;
  k_rows<N, DIR, InSt, OutSt><<<(unsigned)blocks, RowPass<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sense
