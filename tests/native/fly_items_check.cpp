// Host-side check (no GPU) of the local sum with weights computed per pair, traversed as k_local_fly
// traverses it: every item of 32 sources of a spring or receiver row, lanes below the item's real
// source count (item_source_counts), the distance from the positions (periodic minimum image), the
// fitted weights of m >= 1 (local_fit.cuh), summed per row, against the stored FP64 weights (LocalCSR,
// m >= 1) of the same rows.  Input: M R dt tol bc, M positions, R receiver positions.
// Prints "ok <max |difference| / max |row sum|> <items>".
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

static double hist(int m, int64_t l) { return std::sin(0.23 * m + 1.7 * (double)l) + 0.05; }

int main() {
    long M, R;
    double dt, tol;
    int bc;
    if (std::scanf("%ld %ld %lf %lf %d", &M, &R, &dt, &tol, &bc) != 5) return 2;
    std::vector<double> x(M), xr(R), beta(M, 2.0);
    for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : xr) if (std::scanf("%lf", &v) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096, (int64_t)1 << 34,
                             hp, err);
    if (rc == 0) rc = build_receivers(hp, xr.data(), R, err);
    if (rc) { std::printf("error %s\n", err.c_str()); return 1; }
    LocalFit f;
    build_local_fit(hp.P, 7, f);
    const double two_pi = 6.283185307179586476925286766559;
    double worst = 0.0, scale = 0.0;
    auto check = [&](const LocalRows& rows, const LocalItems& items, const LocalCSR& csr, const std::vector<double>& xt,
                     int64_t nrows) {
        std::vector<int8_t> nsrc;
        item_source_counts(rows, items, nsrc);
        std::vector<double> fly(nrows, 0.0);
        for (int64_t o = 0; o < (int64_t)items.row.size(); o++) {
            const int64_t j = items.row[o];
            for (int lane = 0; lane < nsrc[o]; lane++) {
                const int64_t s = items.src[o * 32 + lane];
                double d = std::fabs(xt[j] - hp.x[s]);
                if (bc == WAVE1D_PERIODIC) d = std::min(d, two_pi - d);
                fit::pair_weights(f.bp.data(), (int)f.bp.size() - 1, f.coef.data(), f.mlo.data(), f.mhi.data(), f.deg,
                                  f.nm, d, 1, [&](int m, double q) { fly[j] += q * hist(m, s); });
            }
        }
        for (int64_t j = 0; j < nrows; j++) {
            double stored = 0.0;
            for (int64_t e = csr.row_ptr[j]; e < csr.row_ptr[j + 1]; e++) {
                const int lo = csr.mrange[e] & 0xffff, cnt = csr.mrange[e] >> 16;
                for (int c = 0; c < cnt; c++)
                    if (lo + c >= 1) stored += csr.w[csr.woff[e] + c] * hist(lo + c, csr.src[e]);
            }
            worst = std::max(worst, std::fabs(stored - fly[j]));
            scale = std::max(scale, std::fabs(stored));
        }
        return (int64_t)items.row.size();
    };
    int64_t ni = check(hp.lrows, hp.litems, hp.loc, hp.x, M);
    ni += check(hp.rrows, hp.ritems, hp.rloc, hp.xr, R);
    std::printf("ok %.3e %ld\n", worst / scale, (long)ni);
    return 0;
}
