// Register-FFT axis passes for FFT lengths 1024 and 768.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_1024(X) X(1024, 0) X(768, 0) X(1024, 1) X(1024, 2) X(768, 1) X(1024, 3) X(768, 4)
PSTD_WDISPATCH(w1024, PSTD_WLIST_1024)
}  // namespace pstd
