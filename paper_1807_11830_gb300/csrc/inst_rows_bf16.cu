// Row (x-direction) transform kernels, bf16 storage of k-space.
#include "launch_col.cuh"

namespace sense {

template <>
cudaError_t launch_rows_fwd<StBF16>(int n, const RowArgs<float2, typename StBF16::T>& a, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) case N: return rows_n<N, -1, StC64, StBF16>(a, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_rows_inv<StBF16>(int n, const RowArgs<typename StBF16::T, float2>& a, cudaStream_t s) {
  switch (n) {
#define SENSE_CASE(N) case N: return rows_n<N, 1, StBF16, StC64>(a, s);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sense
