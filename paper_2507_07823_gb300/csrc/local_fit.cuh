// Per-pair evaluation of the piecewise-polynomial local weights (local_fit.h), for both a device
// kernel and host checks: the interval of distance d by bisection over the breakpoints, then the
// Chebyshev series (Clenshaw) of every m >= m_first that is non-zero on that interval.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define WAVE1D_FIT_HD __host__ __device__ __forceinline__
#else
#define WAVE1D_FIT_HD inline
#endif

namespace wave1d {
namespace fit {

// bp[0 .. nint]: breakpoints; coef[(iv nm + m) (deg + 1) + r]; mlo/mhi[iv]: non-zero m range.
// Delivers acc(m, Q_m(d)) for m = max(mlo, m_first) .. mhi; nothing for d outside [0, bp[nint]).
template <class Acc>
WAVE1D_FIT_HD void pair_weights(const double* bp, int nint, const double* coef, const int* mlo, const int* mhi,
                                int deg, int nm, double d, int m_first, Acc acc) {
    if (!(d >= 0.0) || !(d < bp[nint])) return;
    int lo = 0, hi = nint;                         // bp[lo] <= d < bp[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bp[mid] <= d) lo = mid;
        else hi = mid;
    }
    const double z = 2.0 * (d - bp[lo]) / (bp[lo + 1] - bp[lo]) - 1.0;
    const int m0 = mlo[lo] > m_first ? mlo[lo] : m_first;
    for (int m = m0; m <= mhi[lo]; m++) {
        const double* c = coef + ((int64_t)lo * nm + m) * (deg + 1);
        double b0 = 0.0, b1 = 0.0;
        for (int r = deg; r >= 1; r--) {
            const double b2 = b1;
            b1 = b0;
            b0 = 2.0 * z * b1 - b2 + c[r];
        }
        acc(m, z * b0 - b1 + c[0]);
    }
}

}  // namespace fit
}  // namespace wave1d
