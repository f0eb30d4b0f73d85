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
#define SENSE_CASE(N) case N: return Cfg<N>::C::W;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int col_threads(int n) {
  switch (n) {
#define SENSE_CASE(N) case N: return Cfg<N>::C::THREADS;
    SENSE_FOR_EACH_SIZE(SENSE_CASE)
#undef SENSE_CASE
    default:
      return 0;
  }
}

int row_width(int n) { return col_width(n); }

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

}  // namespace sense
