// Persistent CG kernel, bf16 storage of S.
#include "launch_col.cuh"

namespace sense {

template <>
cudaError_t launch_cg_persistent<StBF16>(int n, int variant, const PArgs& a, int sms, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) case N: return persistent_n<N, StBF16>(variant, a, sms, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// blocks per SM of the persistent kernel (StBF16)
int cg_persistent_resident_stbf16(int n, int variant) {
  switch (n) {
#define SENSE_CASE(N) case N: return persistent_resident_n<N, StBF16>(variant);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

}  // namespace sense
