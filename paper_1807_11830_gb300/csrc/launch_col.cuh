// Launcher templates of the column and row kernels (included by the
// per-family instantiation units so the families compile in parallel).
#pragma once
#include "launch.h"

namespace sense {

template <int N, class St>
cudaError_t fwd_col_n(const FwdColArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = col_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_fwd_col<N, St>, sm, &done);
  if (e != cudaSuccess || tiles == 0 || frames == 0) return e;
  k_fwd_col<N, St><<<dim3(tiles, frames), Cfg<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, class St, int MODE>
cudaError_t adj_col_n(const AdjColArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = col_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_adj_col<N, St, MODE>, sm, &done);
  if (e != cudaSuccess || tiles == 0 || frames == 0) return e;
  k_adj_col<N, St, MODE><<<dim3(tiles, frames), Cfg<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, class St, bool CG>
cudaError_t normal_n(const NormalArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = col_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_normal<N, St, CG>, sm, &done);
  if (e != cudaSuccess || tiles == 0 || frames == 0) return e;  // empty grid: attribute set-up only
  k_normal<N, St, CG><<<dim3(tiles, frames), Cfg<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <int N, int DIR, class InSt, class OutSt>
cudaError_t rows_n(const RowArgs<typename InSt::T, typename OutSt::T>& a, cudaStream_t s) {
  static unsigned long long done = 0;
  constexpr size_t sm = row_smem_bytes<N>();
  cudaError_t e = ensure_smem(k_rows<N, DIR, InSt, OutSt>, sm, &done);
  if (e != cudaSuccess) return e;
  const long blocks = (a.rows + Cfg<N>::C::W - 1) / Cfg<N>::C::W;
  if (blocks <= 0) return cudaSuccess;
  k_rows<N, DIR, InSt, OutSt><<<(unsigned)blocks, Cfg<N>::C::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sense
