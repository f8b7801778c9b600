// Local sum (Sec. 4.1) with the weights computed per pair from its distance (plans opened with
// opts.local_weights = 1): the piecewise Chebyshev series of local_fit.h between the rule's
// breakpoints, evaluated by local_fit.cuh, so the device holds no weights.  The work split is the
// stored-weight path's: one warp per item of 32 sources of one row (spring or receiver), lane l
// taking source rank 32 c + l when it is one of the row's real sources (nsrc of the item); each
// item's partial goes to the same slot (l_part / r_part), so the solve and the receivers' readout
// are unchanged.  The distance is recomputed from the positions (the periodic minimum image), the
// density read from the FP64 ring, and the products summed in FP64.  The launch reads the step
// index from the device counter (it sits inside captured step graphs).
#include <cuda_runtime.h>

#include <cstdint>

#include "fly.h"
#include "internal.h"
#include "local_fit.cuh"
#include "phases.cuh"

namespace wave1d {

__device__ __forceinline__ double fly_item(const DevPlan& P, const FlyTables& F, int64_t n, double xt,
                                           const int32_t* src, int nsrc, int lane) {
    if (lane >= nsrc) return 0.0;
    const int64_t s = src[lane];
    double d = fabs(xt - P.x[s]);
    if (P.bc == WAVE1D_PERIODIC) d = fmin(d, 6.283185307179586476925286766559 - d);
    double acc = 0.0;
    fit::pair_weights(F.bp, F.nint, F.coef, F.mlo, F.mhi, F.deg, F.nm, d, 1, [&](int m, double q) {
        acc = fma(q, __ldg(P.sig + (int64_t)ring_slot(n + 1 - m, P.ring) * P.M + s), acc);
    });
    return acc;
}

__global__ void k_local_fly(DevPlan P, FlyTables F) {
    const int lane = threadIdx.x & 31;
    const int64_t n = load_step(P);
    const int64_t total = P.l_nitems + P.r_nitems;
    for (int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < total;
         o += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double v;
        if (o < P.l_nitems) {
            v = fly_item(P, F, n, P.x[P.l_row[o]], P.l_src + o * 32, F.l_nsrc[o], lane);
            v = warp_sum(v);
            if (lane == 0) P.l_part[o] = v;
        } else {
            const int64_t it = o - P.l_nitems;
            // the receiver of item `it`: r_item_ptr[r] <= it < r_item_ptr[r + 1]
            int64_t lo = 0, hi = P.R;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (P.r_item_ptr[mid] <= it) lo = mid;
                else hi = mid;
            }
            v = fly_item(P, F, n, F.xr[lo], P.r_src + it * 32, F.r_nsrc[it], lane);
            v = warp_sum(v);
            if (lane == 0) P.r_part[it] = v;
        }
    }
}

}  // namespace wave1d
