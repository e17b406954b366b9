// Register-FFT axis passes for FFT lengths 2..32.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_SMALL(X) X(2, 0) X(4, 0) X(8, 0) X(16, 0) X(32, 0)
PSTD_WDISPATCH(wsmall, PSTD_WLIST_SMALL)
}  // namespace pstd
