// Host-side check (no GPU) of the local sum of plans without pair lists (opts.local_weights = 1).
//
// Mode "fit": the range tables' polynomials against the plan's own weight rule at random
// distances and every interval's midpoint: prints "ok <intervals> <max err FP64 series> <max err
// of the float-pair monomials>", both relative to max |Q|.
//
// Mode "sum": the local sums c_j = sum_l sum_{m >= 1} Q_m(d_jl) h[m][l] of every spring, once with
// the stored FP64 weights of an ordinary plan and once with the range-mode arithmetic of
// range.cuh driven through the same chunks, interval windows, interval walk and order as the
// k_rs_local kernel (the e-vector of each (source, interval) recomputed per pair, which gives the
// same bits).  Prints "ok <max |difference| / max |row sum|> <pairs>".
//
// Input: mode M dt tol bc, then M positions (mode fit: only dt tol; M positions ignored).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.h"
#include "range.cuh"
#include "wave1d.h"

using namespace wave1d;

static double hist(int m, int64_t l) { return std::cos(0.41 * m + 0.9 * (double)l) + 0.02 * m; }

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

double xext(const HostPlan& hp, int64_t e) {
    const int64_t M = hp.P.M;
    if (e < 0) return hp.x[e + M] - 2.0 * kPi;
    if (e >= M) return hp.x[e - M] + 2.0 * kPi;
    return hp.x[e];
}

rs::Pair xpair(const HostPlan& hp, int64_t e) {
    const int64_t M = hp.P.M, l = e < 0 ? e + M : (e >= M ? e - M : e);
    rs::Pair X{hp.x2[2 * l], hp.x2[2 * l + 1]};
    if (e != l) {
        const float th = (float)(2.0 * kPi), tl = (float)(2.0 * kPi - (double)(float)(2.0 * kPi));
        X = rs::pair_add(X, e < 0 ? rs::Pair{-th, -tl} : rs::Pair{th, tl});
    }
    return X;
}

int locate(const RangeTables& rt, rs::Pair d) {
    int lo = 0, hi = rt.nint;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rs::pair_lt(d, rs::Pair{rt.bp2[2 * mid], rt.bp2[2 * mid + 1]})) hi = mid;
        else lo = mid;
    }
    return lo;
}

void evec_of(const RangeTables& rt, int iv, int64_t l, float* rec) {
    rs::EVec ev;
    rs::evec_zero(ev);
    for (int m = rt.mr[2 * iv]; m <= rt.mr[2 * iv + 1]; m++) {
        const float* c = &rt.coef[((size_t)iv * rt.nm + m) * 12];
        const rs::Pair s = rs::split(hist(m, l));
        rs::evec_mac(ev, c, c + 4, c + 8, s.hi, s.lo);
    }
    const float r[12] = {ev.e0h, ev.e0l, ev.e1h, ev.e1l, ev.e2, ev.e3, ev.e4, ev.e5, ev.e6, ev.e7, 0.f, 0.f};
    std::memcpy(rec, r, sizeof(r));
}

// the kernel's traversal for one block, every target of it
void block_sums(const HostPlan& hp, int64_t b, std::vector<double>& out) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M, j0 = b * kRsTargets;
    const int nT = (int)std::min<int64_t>(kRsTargets, M - j0);
    const int wlo = hp.blk_win[4 * b], inlo = hp.blk_win[4 * b + 1], inhi = hp.blk_win[4 * b + 2],
              whi = hp.blk_win[4 * b + 3];
    const int nL = std::max(0, inhi - wlo), total = nL + std::max(0, whi - inlo);
    const rs::Pair Xa{hp.x2[2 * j0], hp.x2[2 * j0 + 1]};
    const rs::Pair Xb{hp.x2[2 * (j0 + nT - 1)], hp.x2[2 * (j0 + nT - 1) + 1]};
    const rs::Pair zero{0.f, 0.f}, dlim{rt.bp2[2 * rt.nint], rt.bp2[2 * rt.nint + 1]};
    struct T {
        float ah = 0.f, al = 0.f;
        int tiv[2] = {-1, -1};
        rs::Pair Y[2] = {{0.f, 0.f}, {0.f, 0.f}};
    };
    std::vector<T> st(nT);
    const int C = 32, CAP = 32;
    for (int base = 0; base < total; base += C) {
        int sE[32], sLo[32], sHi[32], sType[32];
        rs::Pair sX[32];
        int U0 = INT_MAX, U1 = -1;
        for (int k = 0; k < C; k++) {
            const int v = base + k;
            int lo = 1, hi = 0, type = 0, e = 0;
            rs::Pair X = zero;
            if (v < total) {
                type = v < nL ? 0 : 1;
                e = type == 0 ? wlo + v : inlo + (v - nL);
                X = xpair(hp, e);
                rs::Pair dmin = type == 0 ? rs::pair_sub(Xa, X) : rs::pair_sub(X, Xb);
                rs::Pair dmax = type == 0 ? rs::pair_sub(Xb, X) : rs::pair_sub(X, Xa);
                if (rs::pair_lt(dmin, zero)) dmin = zero;
                if (!rs::pair_lt(dmax, zero) && rs::pair_lt(dmin, dlim)) {
                    lo = std::max(0, rs::locate_tab(rt.bp2.data(), rt.cell.data(), rt.cell_scale, rt.nint, dmin) - 1);
                    hi = std::min(rt.nint - 1, rs::locate_tab(rt.bp2.data(), rt.cell.data(), rt.cell_scale, rt.nint, dmax) + 1);
                }
            }
            sE[k] = e;
            sLo[k] = lo;
            sHi[k] = hi;
            sType[k] = type;
            sX[k] = X;
            if (lo <= hi) {
                U0 = std::min(U0, lo);
                U1 = std::max(U1, hi);
            }
        }
        for (int W0 = U0; W0 <= U1; W0 += CAP) {
            const int W1 = std::min(U1, W0 + CAP - 1);
            for (int t = 0; t < nT; t++) {
                T& s = st[t];
                if (W0 > U0) s.tiv[0] = s.tiv[1] = -1;
                const int64_t j = j0 + t;
                const rs::Pair Xj{hp.x2[2 * j], hp.x2[2 * j + 1]};
                const int nbl = hp.nb_lo[j], nbc = hp.nb_cnt[j];
                const int kend = std::min(C, total - base);
                for (int k = 0; k < kend; k++) {
                    if (sLo[k] > sHi[k]) continue;
                    const int type = sType[k];
                    const rs::Pair X = sX[k];
                    if (type == 0 ? !rs::pair_lt(X, Xj) : rs::pair_lt(X, Xj)) continue;
                    const bool near = (unsigned)(sE[k] - nbl) < (unsigned)nbc;
                    rs::Track tr{s.tiv[type], s.Y[type]};
                    float zh, zl;
                    const bool in = rs::pair_z(rt.bp2.data(), rt.mid2.data(), rt.ih.data(), rt.cell.data(), rt.cell_scale,
                                               rt.nint, rt.iv_dt, type == 0, near, Xj, X, tr, zh, zl);
                    const int iv = tr.iv;
                    s.Y[type] = tr.Y;
                    s.tiv[type] = iv;
                    if (!in) continue;
                    if (iv < W0 || iv > W1 || iv < sLo[k] || iv > sHi[k]) continue;
                    float rec[12];
                    const int64_t l = sE[k] < 0 ? sE[k] + M : (sE[k] >= M ? sE[k] - M : sE[k]);
                    evec_of(rt, iv, l, rec);
                    if (getenv("RS_DEBUG")) fprintf(stderr, "j=%ld e=%d type=%d near=%d iv=%d [%g,%g) z=%g+%g rec0=%g\n", (long)j, sE[k], type, (int)near, iv, rt.bp[iv], rt.bp[iv+1], zh, zl, rec[0]);
                    rs::evec_eval(rec, zh, zl, s.ah, s.al);
                }
            }
        }
    }
    for (int t = 0; t < nT; t++) out[j0 + t] = (double)st[t].ah + (double)st[t].al;
}

}  // namespace

int main() {
    char mode[16];
    long M;
    double dt, tol;
    int bc;
    if (std::scanf("%15s %ld %lf %lf %d", mode, &M, &dt, &tol, &bc) != 5) return 2;
    std::vector<double> x(M), beta(M, 3.0);
    for (auto& v : x)
        if (std::scanf("%lf", &v) != 1) return 2;
    std::string err;
    HostPlan hr;
    if (build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096, (int64_t)1 << 34, hr,
                        err, true)) {
        std::printf("error %s\n", err.c_str());
        return 1;
    }
    const RangeTables& rt = hr.rt;
    if (std::strcmp(mode, "fit") == 0) {
        std::vector<double> d;
        std::mt19937_64 g(7);
        std::uniform_real_distribution<double> u(0.0, hr.P.delta);
        for (int i = 0; i < 4000; i++) d.push_back(u(g));
        for (int iv = 0; iv < rt.nint; iv++) d.push_back(rt.mid[iv]);
        std::vector<double> Q;
        local_weights_exact(hr.P, d, Q);
        const int nm = rt.nm;
        double scale = 0.0, e64 = 0.0, e32 = 0.0;
        for (size_t i = 0; i < d.size(); i++) {
            int iv = (int)(std::upper_bound(rt.bp.begin(), rt.bp.end(), d[i]) - rt.bp.begin()) - 1;
            iv = std::min(std::max(iv, 0), rt.nint - 1);
            const double z = (d[i] - rt.mid[iv]) * (double)rt.ih[iv];
            for (int m = 0; m < nm; m++) {
                const double* c = &rt.cheb[((size_t)iv * nm + m) * 8];
                double b0 = 0.0, b1 = 0.0;
                for (int r = 7; r >= 1; r--) {
                    const double b2 = b1;
                    b1 = b0;
                    b0 = 2.0 * z * b1 - b2 + c[r];
                }
                const double q64 = z * b0 - b1 + c[0];
                const float* a = &rt.coef[((size_t)iv * nm + m) * 12];
                double q32 = 0.0;
                for (int r = 7; r >= 4; r--) q32 = q32 * z + (double)a[4 + r];
                for (int r = 3; r >= 0; r--) q32 = q32 * z + ((double)a[2 * r] + (double)a[2 * r + 1]);
                const double q = Q[i * nm + m];
                scale = std::max(scale, std::fabs(q));
                e64 = std::max(e64, std::fabs(q64 - q));
                e32 = std::max(e32, std::fabs(q32 - q));
            }
        }
        std::printf("ok %d %.3e %.3e\n", rt.nint, e64 / scale, e32 / scale);
        return 0;
    }
    HostPlan hs;
    if (build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, 8, 0.5, 0, 0, 32, 0, 0, 4096, (int64_t)1 << 34, hs,
                        err)) {
        std::printf("error %s\n", err.c_str());
        return 1;
    }
    std::vector<double> ref(M, 0.0), got(M, 0.0);
    const LocalCSR& Cs = hs.loc;
    for (int64_t j = 0; j < M; j++)
        for (int64_t e = Cs.row_ptr[j]; e < Cs.row_ptr[j + 1]; e++) {
            const int lo = Cs.mrange[e] & 0xffff, cnt = Cs.mrange[e] >> 16;
            for (int c = 0; c < cnt; c++) ref[j] += Cs.w[Cs.woff[e] + c] * hist(lo + c, Cs.src[e]);
        }
    const int64_t nblk = (M + kRsTargets - 1) / kRsTargets;
    for (int64_t b = 0; b < nblk; b++) block_sums(hr, b, got);
    double worst = 0.0, scale = 0.0;
    for (int64_t j = 0; j < M; j++) {
        worst = std::max(worst, std::fabs(got[j] - ref[j]));
        scale = std::max(scale, std::fabs(ref[j]));
    }
    (void)xext;
    std::printf("ok %.3e %zu\n", worst / scale, Cs.src.size());
    return 0;
}
