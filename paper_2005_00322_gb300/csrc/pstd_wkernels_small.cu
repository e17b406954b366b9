// Register-FFT axis passes for FFT lengths 2..256 and 96, 192.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_SMALL(X) X(2, 0) X(4, 0) X(8, 0) X(16, 0) X(32, 0) X(64, 0) X(128, 0) X(256, 0) X(96, 0) X(192, 0) X(256, 1) X(256, 4) X(256, 5)
PSTD_WDISPATCH(wsmall, PSTD_WLIST_SMALL)
}  // namespace pstd
