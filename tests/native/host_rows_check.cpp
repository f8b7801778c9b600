// Host-side check of the local-sum tables (no GPU): builds the plan tables for a layout read from
// stdin and compares, row by row, the local sum sum_l sum_{m>=1} Q_m(d_jl) h[m][l] for a fixed
// pseudo-random history h computed three ways: from the weight table (CSR), from the m-ordered
// rows, and from the 32-source work items the step kernel reads.  Prints the worst relative
// difference.  Input: M dt tol bc R, then M positions, M stiffnesses and R receiver positions; the
// receivers' tables (m >= 0) are checked the same way.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    long M, R;
    double dt, tol;
    int bc;
    if (std::scanf("%ld %lf %lf %d %ld", &M, &dt, &tol, &bc, &R) != 5) return 2;
    std::vector<double> x(M), beta(M), xr(R);
    for (long j = 0; j < M; j++) if (std::scanf("%lf", &x[j]) != 1) return 2;
    for (long j = 0; j < M; j++) if (std::scanf("%lf", &beta[j]) != 1) return 2;
    for (long j = 0; j < R; j++) if (std::scanf("%lf", &xr[j]) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096,
                             (int64_t)1 << 34, hp, err);
    if (rc == 0 && R > 0) rc = build_receivers(hp, xr.data(), R, err);
    if (rc) {
        std::printf("error %d %s\n", rc, err.c_str());
        return 1;
    }
    const int mm = hp.P.m_max;
    std::vector<double> h((size_t)(mm + 1) * M);
    unsigned long long s = 88172645463325252ull;          // xorshift64
    for (auto& v : h) {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        v = (double)(s >> 11) / 9007199254740992.0 - 0.5;
    }
    // rows and items hold m >= 1 (the m = 0 weights of nearby springs live in the implicit blocks,
    // those of receivers in a separate list applied once sigma^{n+1} is known)
    auto check = [&](const LocalCSR& L, const LocalRows& Rw, const LocalItems& I, long T) {
        double worst = 0.0;
        for (long j = 0; j < T; j++) {
            double a = 0.0, b = 0.0, c = 0.0, scale = 0.0;
            for (int64_t q = L.row_ptr[j]; q < L.row_ptr[j + 1]; q++) {
                const int lo = L.mrange[q] & 0xffff, cnt = L.mrange[q] >> 16;
                for (int m = std::max(lo, 1); m < lo + cnt; m++) {
                    const double t = L.w[L.woff[q] + m - lo] * h[(size_t)m * M + L.src[q]];
                    a += t;
                    scale += std::fabs(t);
                }
            }
            int64_t off = Rw.w_off[j];
            for (int i = 0; i < Rw.nm; i++) {
                const int cn = Rw.cnt[(size_t)j * Rw.nm + i];
                for (int r = 0; r < cn; r++) {
                    const double wv = (double)Rw.w[2 * (off + r)] + (double)Rw.w[2 * (off + r) + 1];
                    b += wv * h[(size_t)(Rw.m_first + i) * M + Rw.src[Rw.src_off[j] + r]];
                }
                off += cn;
            }
            for (int64_t it = I.item_ptr[j]; it < I.item_ptr[j + 1]; it++)
                for (int l = 0; l < 32; l++)
                    for (int t = 0; t < I.len[it]; t++) {
                        const int64_t k = I.wbase[it] + 64 * (int64_t)(t >> 1) + 2 * l + (t & 1);
                        const double wv = (double)I.w[2 * k] + (double)I.w[2 * k + 1];
                        const int m = I.m_first + I.s0[it] + t;
                        if (wv != 0.0 && m <= mm) c += wv * h[(size_t)m * M + I.src[it * 32 + l]];
                    }
            if (scale > 0.0) worst = std::fmax(worst, std::fmax(std::fabs(a - b), std::fabs(a - c)) / scale);
        }
        return worst;
    };
    double worst = check(hp.loc, hp.lrows, hp.litems, M);
    if (R > 0) {
        worst = std::fmax(worst, check(hp.rloc, hp.rrows, hp.ritems, R));
        // the receivers' m = 0 list against the table's m = 0 weights
        for (long r = 0; r < R; r++) {
            double a = 0.0, b = 0.0, scale = 0.0;
            for (int64_t q = hp.rloc.row_ptr[r]; q < hp.rloc.row_ptr[r + 1]; q++) {
                const int lo = hp.rloc.mrange[q] & 0xffff, cnt = hp.rloc.mrange[q] >> 16;
                if (lo == 0 && cnt > 0) {
                    a += hp.rloc.w[hp.rloc.woff[q]] * h[hp.rloc.src[q]];
                    scale += std::fabs(hp.rloc.w[hp.rloc.woff[q]] * h[hp.rloc.src[q]]);
                }
            }
            for (int64_t e = hp.r0_ptr[r]; e < hp.r0_ptr[r + 1]; e++) b += hp.r0_w[e] * h[hp.r0_src[e]];
            if (scale > 0.0) worst = std::fmax(worst, std::fabs(a - b) / scale);
        }
    }
    std::printf("%.6e\n", worst);
    return 0;
}
