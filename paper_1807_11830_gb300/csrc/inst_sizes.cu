// Size table queries (host).
#include "launch_col.cuh"

namespace sense {

bool size_supported(int n) {
  switch (n) {
#define SENSE_CASE(N) case N:
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    return true;
    default:
      return false;
  }
}

int col_width(int n) {
  switch (n) {
#define SENSE_CASE(N) case N: return ColPass<N>::C::W;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int col_threads(int n) {
  switch (n) {
#define SENSE_CASE(N) case N: return ColPass<N>::C::THREADS;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int row_width(int n) {
  switch (n) {
#define SENSE_CASE(N) case N: return RowPass<N>::C::W;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int normal_variant_threads(int n, int variant) {
  switch (n) {
#define SENSE_CASE(N) case N: return norm_variant_threads<N>(variant);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int normal_variant_width(int n, int variant) {
  switch (n) {
#define SENSE_CASE(N) case N: return norm_variant_width<N>(variant);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int normal_variant_transposed(int n, int variant) {
  switch (n) {
#define SENSE_CASE(N) case N: return norm_variant_transposed<N>(variant);
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

template <class E>
static cudaError_t transpose_maps(const E* S, E* ST, int ny, int nx, int coils, cudaStream_t s) {
  if (coils == 0) return cudaSuccess;
  const dim3 grid((nx + 31) / 32, (ny + 31) / 32, coils);
  k_transpose_maps<E><<<grid, dim3(32, 8), 0, s>>>(S, ST, ny, nx);
  return cudaGetLastError();
}

cudaError_t launch_transpose_maps(bool bf16, const void* S, void* ST, int ny, int nx, int coils, cudaStream_t s) {
  if (bf16)
    return transpose_maps(static_cast<const __nv_bfloat162*>(S), static_cast<__nv_bfloat162*>(ST), ny, nx, coils, s);
  return transpose_maps(static_cast<const float2*>(S), static_cast<float2*>(ST), ny, nx, coils, s);
}

}  // namespace sense

namespace sense {

int cg_persistent_resident_stc64(int n, int variant);
int cg_persistent_resident_stbf16(int n, int variant);

int cg_persistent_resident(int n, int variant, bool bf16) {
  return bf16 ? cg_persistent_resident_stbf16(n, variant) : cg_persistent_resident_stc64(n, variant);
}

}  // namespace sense
