// Host-side check of the local-sum tables (no GPU): builds the plan tables for a layout read from
// stdin and compares, row by row, the local sum sum_l sum_{m>=1} Q_m(d_jl) h[m][l] for a fixed
// pseudo-random history h computed three ways: from the weight table (CSR), from the m-ordered
// rows, and from the 32-source work items the step kernel reads.  Prints the worst relative
// difference.  Input: M dt tol bc, then M positions and M stiffnesses.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    long M;
    double dt, tol;
    int bc;
    if (std::scanf("%ld %lf %lf %d", &M, &dt, &tol, &bc) != 4) return 2;
    std::vector<double> x(M), beta(M);
    for (long j = 0; j < M; j++) if (std::scanf("%lf", &x[j]) != 1) return 2;
    for (long j = 0; j < M; j++) if (std::scanf("%lf", &beta[j]) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096,
                             (int64_t)1 << 34, hp, err);
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
    const LocalCSR& L = hp.loc;
    const LocalRows& R = hp.lrows;
    const LocalItems& I = hp.litems;
    double worst = 0.0;
    for (long j = 0; j < M; j++) {
        double a = 0.0, b = 0.0, c = 0.0, scale = 0.0;
        for (int64_t q = L.row_ptr[j]; q < L.row_ptr[j + 1]; q++) {
            const int lo = L.mrange[q] & 0xffff, cnt = L.mrange[q] >> 16;
            for (int m = lo; m < lo + cnt; m++) {
                const double t = L.w[L.woff[q] + m - lo] * h[(size_t)m * M + L.src[q]];
                a += t;
                scale += std::fabs(t);
            }
        }
        int64_t off = R.w_off[j];
        for (int i = 0; i < R.nm; i++) {
            const int cn = R.cnt[(size_t)j * R.nm + i];
            for (int r = 0; r < cn; r++) {
                const double wv = (double)R.w[2 * (off + r)] + (double)R.w[2 * (off + r) + 1];
                b += wv * h[(size_t)(R.m_first + i) * M + R.src[R.src_off[j] + r]];
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
    std::printf("%.6e\n", worst);
    return 0;
}
