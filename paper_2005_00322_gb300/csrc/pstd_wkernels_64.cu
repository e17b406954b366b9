// Register-FFT axis passes for FFT lengths 64, 128, 96 and 192.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_64(X) X(64, 0) X(128, 0) X(96, 0) X(192, 0)
PSTD_WDISPATCH(w64, PSTD_WLIST_64)
}  // namespace pstd
