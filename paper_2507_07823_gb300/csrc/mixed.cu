// Mixed-precision history part of the time step (plans opened with opts.precision = 1): the
// type-1 spreading and type-2 interpolation of the step (eq. densco, eq. historySol1) run through
// the FP32 NUFFT kernels of csrc/nufft.cu on the plan's springs (and receivers); the FFTs, the
// mode recurrence, the local sum and the density solve stay as in the FP64 step.  These launches
// sit inside the step's captured graphs, so they read the step index from the device counter.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phases.cuh"

namespace wave1d {

// c[i] = sigma^n of spring perm[i] (the NUFFT plan's point order)
__global__ void k_mx_gather(DevPlan P, const int64_t* __restrict__ perm, double* __restrict__ c) {
    const int64_t n = load_step(P);
    const double* sg = P.sig + (int64_t)ring_slot(n, P.ring) * P.M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = sg[perm[i]];
}

// u_H at spring perm[i] and the u_H part of the right-hand side of eq. linearSystem,
// rhs_j = -g_j(t_{n+1}) - beta_j u_H(x_j), as the FP64 interpolation forms them
__global__ void k_mx_rhs(DevPlan P, const int64_t* __restrict__ perm, const double* __restrict__ u) {
    const int64_t n = load_step(P);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = perm[i];
        const double uh = u[i];
        P.uH[j] = uh;
        P.rhs[j] = -forcing(P, n, j) - P.beta[j] * uh;
    }
}

// u_H at receiver perm[i]
__global__ void k_mx_receivers(int64_t R, const int64_t* __restrict__ perm, const double* __restrict__ u,
                               double* __restrict__ uHr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R; i += (int64_t)gridDim.x * blockDim.x)
        uHr[perm[i]] = u[i];
}

}  // namespace wave1d
