// pstd_energy.h -- FP64 discrete energy of the leapfrog state (pstd_energy.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pstd {

// One field's sum_j w_j a_j b_j over an n[0] x n[1] x n[2] array (C order);
// bit a of first_half / last_half halves the weight of index 0 / n[a] - 1
// along axis a.
struct EnergyField {
    const float* a;
    const float* b;
    int64_t n[3];
    int first_half, last_half;
};

struct EnergyScales {
    double s[4];
};

// Partial sums of every field into scratch[f * nblocks + block], then
// scratch[4 * nblocks] = sum_f s[f] * (field f's sum).  scratch holds at least
// 4 * nblocks + 1 doubles.
cudaError_t energy_launch(const EnergyField* fields, int nfields, const EnergyScales& sc, int nblocks,
                          double* scratch, cudaStream_t st);

}  // namespace pstd
