// Host-side check (no GPU) of local sums from weights computed per pair (local_fit.cuh) against the
// plan's stored FP64 weights (LocalCSR, m >= 1): for every spring row j,
//   sum_{l in row j} sum_{m >= 1} Q_m(d_jl) h[m][l]
// with Q_m from the stored table and from the degree-deg fit at d_jl recomputed from the positions
// (the periodic minimum image where the box is periodic).  Input: M dt tol bc deg, then M positions.
// Prints "ok <max |difference| / max |row sum|> <pairs>".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "local_fit.cuh"
#include "local_fit.h"
#include "wave1d.h"

using namespace wave1d;

static double hist(int m, int64_t l) { return std::cos(0.41 * m + 0.9 * (double)l) + 0.02 * m; }

int main() {
    long M;
    double dt, tol;
    int bc, deg;
    if (std::scanf("%ld %lf %lf %d %d", &M, &dt, &tol, &bc, &deg) != 5) return 2;
    std::vector<double> x(M), beta(M, 3.0);
    for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
    HostPlan hp;
    std::string err;
    if (build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096, (int64_t)1 << 34, hp,
                        err)) {
        std::printf("error %s\n", err.c_str());
        return 1;
    }
    LocalFit f;
    build_local_fit(hp.P, deg, f);
    const LocalCSR& C = hp.loc;
    const double two_pi = 6.283185307179586476925286766559;
    double worst = 0.0, scale = 0.0;
    for (int64_t j = 0; j < M; j++) {
        double stored = 0.0, fitted = 0.0;
        for (int64_t e = C.row_ptr[j]; e < C.row_ptr[j + 1]; e++) {
            const int64_t l = C.src[e];
            const int lo = C.mrange[e] & 0xffff, cnt = C.mrange[e] >> 16;
            for (int c = 0; c < cnt; c++) stored += C.w[C.woff[e] + c] * hist(lo + c, l);
            double d = std::fabs(hp.x[j] - hp.x[l]);
            if (bc == WAVE1D_PERIODIC) d = std::min(d, two_pi - d);
            fit::pair_weights(f.bp.data(), (int)f.bp.size() - 1, f.coef.data(), f.mlo.data(), f.mhi.data(), f.deg,
                              f.nm, d, 1, [&](int m, double q) { fitted += q * hist(m, l); });
        }
        worst = std::max(worst, std::fabs(stored - fitted));
        scale = std::max(scale, std::fabs(stored));
    }
    std::printf("ok %.3e %zu\n", worst / scale, C.src.size());
    return 0;
}
