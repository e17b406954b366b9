// Register-FFT axis passes for FFT length 1024, the throughput schedules.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_1024T(X) X(1024, 0) X(1024, 2)
PSTD_WDISPATCH(w1024t, PSTD_WLIST_1024T)
}  // namespace pstd
