// Register-FFT axis passes for FFT length 512.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_512(X) X(512, 0) X(512, 1) X(512, 3) X(512, 4) X(512, 5)
PSTD_WDISPATCH(w512, PSTD_WLIST_512)
}  // namespace pstd
