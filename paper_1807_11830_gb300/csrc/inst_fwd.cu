// E column kernels, both storages of S.
#include "launch_col.cuh"

namespace sense {

template <class St>
static cudaError_t fwd_dispatch(int n, const FwdColArgs<St>& a, int tiles, int frames, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) case N: return fwd_col_n<N, St>(a, tiles, frames, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_fwd_col<StC64>(int n, const FwdColArgs<StC64>& a, int tiles, int frames, cudaStream_t s) {
  return fwd_dispatch<StC64>(n, a, tiles, frames, s);
}

template <>
cudaError_t launch_fwd_col<StBF16>(int n, const FwdColArgs<StBF16>& a, int tiles, int frames, cudaStream_t s) {
  return fwd_dispatch<StBF16>(n, a, tiles, frames, s);
}

}  // namespace sense
