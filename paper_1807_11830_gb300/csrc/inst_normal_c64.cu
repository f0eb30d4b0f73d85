// E^H E column kernels, c64 storage of S.
#include "launch_col.cuh"

namespace sense {

template <>
cudaError_t launch_normal<StC64>(int n, int variant, bool cg, const NormalArgs<StC64>& a, int frames,
                                cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) \
  case N:             \
    return cg ? normal_n<N, StC64, true>(variant, a, frames, s) : normal_n<N, StC64, false>(variant, a, frames, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sense
