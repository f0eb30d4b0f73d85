// Size table queries (host).
#include "launch.h"

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

}  // namespace sense
