// Register-FFT axis passes for FFT length 256.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_256(X) X(256, 0) X(256, 1) X(256, 4) X(256, 5)
PSTD_WDISPATCH(w256, PSTD_WLIST_256)
}  // namespace pstd
