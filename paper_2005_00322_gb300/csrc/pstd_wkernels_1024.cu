// Register-FFT axis passes for FFT length 1024, the latency schedules.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_1024(X) X(1024, 1) X(1024, 3)
PSTD_WDISPATCH(w1024, PSTD_WLIST_1024)
}  // namespace pstd
