// Standalone kernels of the history pipeline (one launch per phase; see phases.cuh for what each
// phase computes).  On projection steps k_hist_rows stops after the mode update and the
// natural-order inverse FFT of the projected spectrum runs instead of k_hist_icols.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phases.cuh"

namespace wave1d {

__global__ void k_hist_cols(DevPlan P, double2* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cols_phase(P, load_step(P), Y, blockIdx.x, smraw);
}

__global__ void k_hist_rows(DevPlan P, const double2* __restrict__ Y, double2* __restrict__ T, int do_inverse) {
    extern __shared__ __align__(16) unsigned char smraw[];
    rows_phase(P, load_step(P), Y, T, blockIdx.x, do_inverse, smraw);
}

// FIR tail of the step (before the rows), kTailModes modes per block (256 threads)
__global__ void k_hist_tail(DevPlan P) {
    const int k = blockIdx.x * kTailModes + (int)(threadIdx.x >> 3);
    fir_tail(P, load_step(P), k, k <= P.K);
}

__global__ void k_hist_icols(DevPlan P, const double2* __restrict__ T) {
    extern __shared__ __align__(16) unsigned char smraw[];
    icols_phase(P, T, blockIdx.x, smraw);
}

}  // namespace wave1d
