// E^H column kernels (adjoint, CG start, root sum of squares), c64 storage of S.
#include "launch_col.cuh"

namespace sense {

template <>
cudaError_t launch_adj_col<StC64>(int n, int mode, const AdjColArgs<StC64>& a, int tiles, int frames,
                                 cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N)                                                     \
  case N:                                                                 \
    if (mode == 0) return adj_col_n<N, StC64, 0>(a, tiles, frames, s);   \
    if (mode == 1) return adj_col_n<N, StC64, 1>(a, tiles, frames, s);   \
    if (mode == 2) return adj_col_n<N, StC64, 2>(a, tiles, frames, s); \
    return cudaErrorInvalidValue;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sense
