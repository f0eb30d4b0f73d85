// Persistent CG kernel, c64 storage of S.
#include "launch_col.cuh"

namespace sense {

template <>
cudaError_t launch_cg_persistent<StC64>(int n, int variant, const PArgs& a, int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) case N: return persistent_n<N, StC64>(variant, a, sms, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// blocks per SM of the persistent kernel (StC64)
int cg_persistent_resident_stc64(int n, int variant) {
  switch (n) {
#define SENSE_CASE(N) case N: return persistent_resident_n<N, StC64>(variant);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

}  // namespace sense
