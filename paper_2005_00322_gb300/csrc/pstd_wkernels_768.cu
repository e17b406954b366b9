// Register-FFT axis passes for FFT lengths 768 and 384.
#include <cmath>
#include "pstd_wkernels.cuh"
namespace pstd {
#define PSTD_WLIST_768(X) X(768, 0) X(768, 1) X(768, 4) X(384, 0)
PSTD_WDISPATCH(w768, PSTD_WLIST_768)
}  // namespace pstd
