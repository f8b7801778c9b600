// Host-side check (no GPU) of the local sum of plans without pair lists (opts.local_weights = 1).
//
// Mode "fit": the range tables' polynomials against the plan's own weight rule at random
// distances and every interval's midpoint: prints "ok <intervals> <max err FP64 series> <max err
// of the float-pair monomials>", both relative to max |Q|.
//
// Mode "sum": the local sums c_j = sum_l sum_{m >= 1} Q_m(d_jl) h[m][l] of every spring, once with
// the stored FP64 weights of an ordinary plan and once with the range-mode arithmetic of
// range.cuh driven through the same chunks, interval windows (or, in chunks with few pairs per
// e-vector, one pass per pair; in blocks whose targets lie farther apart than two window widths,
// each target's own sources), interval walk and order as the k_rs_local kernel (the e-vector of
// each (source, interval) recomputed per pair, which gives the same bits).  Prints "ok <max |difference| / max |row sum|> <pairs>".
//
// Mode "tsum": the reverse march's transposed local sums out_j[m] = sum_e Q_m(d_je) cbar_e, m >= 1,
// through the k_rs_local_T kernel's traversal (per output: the forward block's window in order,
// the moments of the current interval flushed into out[m] when the interval changes) against the
// stored FP64 weights.  Prints "ok <max |difference| / max |out|> <pairs>".
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

// the pairs of one side for one target, sources [k0, k1) of the chunk (rs_pairs of the kernel)
template <int S>
void side_pairs(const HostPlan& hp, const std::vector<float>& ivt, const float* meta, int k0, int k1, int W0, int W1,
                int64_t lbj, int nbl, int nbc, float bh, float bl, rs::Track& tr, float acc[4]) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M;
    for (int k = k0; k < k1; k++) {
        const float* mt = meta + 4 * k;
        int e, lohi;
        std::memcpy(&e, mt + 2, 4);
        std::memcpy(&lohi, mt + 3, 4);
        const int lo = std::max(lohi & 0x7fff, W0), hi = std::min(lohi >> 16, W1);
        if (lo > hi || (S < 0 ? e >= lbj : e < lbj)) continue;
        float zh, zl;
        rs::z_of<S>(tr, mt[0], mt[1], zh, zl);
        if (std::fabs(zh) > rs::kZTol)
            rs::walk<S>(ivt.data(), rt.cell.data(), rt.cell_scale, rt.nint, bh, bl, mt[0], mt[1], tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt.data(), rt.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt[0], mt[1], tr, zh,
                             zl);
        if (!(std::fabs(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi)) continue;
        float rec[12];
        const int64_t l = e < 0 ? e + M : (e >= M ? e - M : e);
        evec_of(rt, tr.iv, l, rec);
        float* a = acc + 2 * (k & 1);
        rs::evec_eval(rec, zh, zl, a[0], a[1]);
    }
}

// a chunk of several windows: the sources of one side in walk order from the cursor, each walked
// once (the kernel's rs_pairs_cursor)
template <int S>
void cursor_pairs(const HostPlan& hp, const std::vector<float>& ivt, const float* meta, int k0, int k1, int& cur,
                  int W0, int W1, int64_t lbj, int nbl, int nbc, float bh, float bl, rs::Track& tr, int& par,
                  float acc[4]) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M;
    while (S > 0 ? cur < k1 : cur >= k0) {
        const int k = cur;
        const float* mt = meta + 4 * k;
        int e, lohi;
        std::memcpy(&e, mt + 2, 4);
        std::memcpy(&lohi, mt + 3, 4);
        const int lo = lohi & 0x7fff, hi = lohi >> 16;
        if (lo > hi || (S < 0 ? e >= lbj : e < lbj)) {
            cur += S;
            continue;
        }
        if (lo > W1) break;
        float zh, zl;
        rs::z_of<S>(tr, mt[0], mt[1], zh, zl);
        if (std::fabs(zh) > rs::kZTol)
            rs::walk<S>(ivt.data(), rt.cell.data(), rt.cell_scale, rt.nint, bh, bl, mt[0], mt[1], tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt.data(), rt.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt[0], mt[1], tr, zh,
                             zl);
        if (tr.iv > W1 && std::fabs(zh) <= rs::kZTol) break;
        if (std::fabs(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi && tr.iv >= W0) {
            float rec[12];
            evec_of(rt, tr.iv, e < 0 ? e + M : (e >= M ? e - M : e), rec);
            float* a = acc + 2 * par;
            rs::evec_eval(rec, zh, zl, a[0], a[1]);
            par ^= 1;
        } else if (zh > rs::kZTol && tr.iv == rt.nint - 1) {
            cur = S > 0 ? k1 : k0 - 1;
            break;
        }
        cur += S;
    }
}

// a chunk where the kernel folds one e-vector per pair: sources [k0, k1) once, no windows
template <int S>
void direct_pairs(const HostPlan& hp, const std::vector<float>& ivt, const float* meta, int k0, int k1, int64_t lbj,
                  int nbl, int nbc, float bh, float bl, rs::Track& tr, float acc[4]) {
    side_pairs<S>(hp, ivt, meta, k0, k1, 0, INT_MAX, lbj, nbl, nbc, bh, bl, tr, acc);
}

// a block whose targets lie farther apart than two window widths: each target walks its own
// sources nearest first on one side until they lie beyond delta (the kernel's sparse-block path)
template <int S>
void sparse_side(const HostPlan& hp, const std::vector<float>& ivt, rs::Grid G, double xa, double span, int64_t j,
                 int wlo, int whi, int64_t lbj, float bh, float bl, rs::Track& tr, float acc[4]) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M;
    const double xj = hp.x[j], reach = hp.P.delta * (1.0 + 8.0 * rs::kRangeMargin);
    const int nbl = hp.nb_lo[j], nbc = hp.nb_cnt[j];
    for (int q = 0;; q++) {
        const int64_t e = S > 0 ? lbj + q : lbj - 1 - q;
        if (S > 0 ? e >= whi : e < wlo) break;
        const double xe = xext(hp, e);
        if (!((S > 0 ? xe - xj : xj - xe) < reach)) break;
        const double xr = xe - xa;
        const int lohi = rs::source_range(xr, S < 0, span, hp.P.delta, hp.P.dt, rt.bp2.data(), rt.cell.data(),
                                          rt.cell_scale, rt.nint);
        const int lo = lohi & 0x7fff, hi = lohi >> 16;
        if (lo > hi) continue;
        float h, l;
        rs::grid_split(xr, G, h, l);
        float zh, zl;
        rs::z_of<S>(tr, h, l, zh, zl);
        if (std::fabs(zh) > rs::kZTol)
            rs::walk<S>(ivt.data(), rt.cell.data(), rt.cell_scale, rt.nint, bh, bl, h, l, tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt.data(), rt.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, h, l, tr, zh, zl);
        if (!(std::fabs(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi)) continue;
        float rec[12];
        evec_of(rt, tr.iv, e < 0 ? e + M : (e >= M ? e - M : e), rec);
        float* a = acc + 2 * (q & 1);
        rs::evec_eval(rec, zh, zl, a[0], a[1]);
    }
}

// the kernel's traversal for one block, every target of it
void block_sums(const HostPlan& hp, int64_t b, std::vector<double>& out) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M, j0 = b * kRsTargets;
    const int nT = (int)std::min<int64_t>(kRsTargets, M - j0);
    const int wlo = hp.blk_win[4 * b], inlo = hp.blk_win[4 * b + 1], inhi = hp.blk_win[4 * b + 2],
              whi = hp.blk_win[4 * b + 3];
    const int nL = std::max(0, inhi - wlo), total = nL + std::max(0, whi - inlo);
    const double xa = hp.x[j0], span = hp.x[j0 + nT - 1] - xa;
    const rs::Grid G = rs::grid_of(span, hp.P.delta);
    std::vector<float> ivt(4 * (size_t)rt.nint);
    for (int iv = 0; iv < rt.nint; iv++) rs::interval_on_grid(rt.mid[iv], rt.ih[iv], G, &ivt[4 * (size_t)iv]);
    struct T {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        float hj = 0.f, lj = 0.f;
        int64_t lbj = 0;
        rs::Track trL{}, trR{};
    };
    std::vector<T> st(nT);
    std::vector<float> sT(nT);
    for (int t = 0; t < nT; t++) sT[t] = (float)(hp.x[j0 + t] - xa);
    for (int t = 0; t < nT; t++) {
        const int64_t j = j0 + t;
        rs::grid_split(hp.x[j] - xa, G, st[t].hj, st[t].lj);
        int64_t lbj = j;
        while (lbj > 0 && hp.x[lbj - 1] == hp.x[j]) lbj--;
        st[t].lbj = lbj;
        rs::track_to(ivt.data(), 0, st[t].hj, st[t].lj, st[t].trL);
        rs::track_to(ivt.data(), 0, -st[t].hj, -st[t].lj, st[t].trR);
    }
    if (span > 2.0 * hp.P.delta) {
        for (int t = 0; t < nT; t++) {
            T& s = st[t];
            sparse_side<-1>(hp, ivt, G, xa, span, j0 + t, wlo, whi, s.lbj, s.hj, s.lj, s.trL, s.acc);
            sparse_side<1>(hp, ivt, G, xa, span, j0 + t, wlo, whi, s.lbj, -s.hj, -s.lj, s.trR, s.acc);
            out[j0 + t] = ((double)s.acc[0] + (double)s.acc[1]) + ((double)s.acc[2] + (double)s.acc[3]);
        }
        return;
    }
    const int C = 32, CAP = 32;
    for (int base = 0; base < total; base += C) {
        float meta[4 * 32];
        int U0 = INT_MAX, U1 = -1, pairs_est = 0;
        for (int k = 0; k < C; k++) {
            const int v = base + k;
            int lohi = 1, e = 0;
            float h = 0.f, l = 0.f;
            if (v < total) {
                const bool left = v < nL;
                e = left ? wlo + v : inlo + (v - nL);
                const double xr = xext(hp, e) - xa;
                rs::grid_split(xr, G, h, l);
                lohi = rs::source_range(xr, left, span, hp.P.delta, hp.P.dt, rt.bp2.data(), rt.cell.data(),
                                        rt.cell_scale, rt.nint);
            }
            const int lo = lohi & 0x7fff, hi = lohi >> 16;
            meta[4 * k] = h;
            meta[4 * k + 1] = l;
            std::memcpy(&meta[4 * k + 2], &e, 4);
            std::memcpy(&meta[4 * k + 3], &lohi, 4);
            if (lo <= hi) {
                U0 = std::min(U0, lo);
                U1 = std::max(U1, hi);
                // the kernel's estimate of the source's targets within delta (float positions)
                const float xf = (float)(xext(hp, e) - xa), df = (float)hp.P.delta;
                const int a = (int)(std::upper_bound(sT.begin(), sT.end(), xf - df) - sT.begin());
                const int c = (int)(std::lower_bound(sT.begin() + a, sT.end(), xf + df) - sT.begin());
                pairs_est += c - a;
            }
        }
        const int kend = std::min(C, total - base), kL = std::min(kend, std::max(0, nL - base));
        if (U1 >= U0 && 2 * pairs_est < C * (U1 - U0 + 1)) {
            for (int t = 0; t < nT; t++) {
                T& s = st[t];
                const int64_t j = j0 + t;
                direct_pairs<-1>(hp, ivt, meta, 0, kL, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], s.hj, s.lj, s.trL, s.acc);
                direct_pairs<1>(hp, ivt, meta, kL, kend, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], -s.hj, -s.lj, s.trR, s.acc);
            }
            continue;
        }
        const bool multi = U1 - U0 + 1 > CAP;
        std::vector<int> curL(nT, kL - 1), curR(nT, kL), par(nT, 0);
        for (int W0 = U0; W0 <= U1; W0 += CAP) {
            const int W1 = std::min(U1, W0 + CAP - 1);
            for (int t = 0; multi && t < nT; t++) {
                T& s = st[t];
                const int64_t j = j0 + t;
                cursor_pairs<-1>(hp, ivt, meta, 0, kL, curL[t], W0, W1, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], s.hj, s.lj, s.trL,
                                 par[t], s.acc);
                cursor_pairs<1>(hp, ivt, meta, kL, kend, curR[t], W0, W1, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], -s.hj, -s.lj,
                                s.trR, par[t], s.acc);
            }
            for (int t = 0; !multi && t < nT; t++) {
                T& s = st[t];
                const int64_t j = j0 + t;
                side_pairs<-1>(hp, ivt, meta, 0, kL, W0, W1, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], s.hj, s.lj, s.trL, s.acc);
                side_pairs<1>(hp, ivt, meta, kL, kend, W0, W1, s.lbj, hp.nb_lo[j], hp.nb_cnt[j], -s.hj, -s.lj, s.trR,
                              s.acc);
            }
        }
    }
    for (int t = 0; t < nT; t++)
        out[j0 + t] = ((double)st[t].acc[0] + (double)st[t].acc[1]) + ((double)st[t].acc[2] + (double)st[t].acc[3]);
}

// ---- transposed local sum (the reverse march's k_rs_local_T): out_j[m] = sum_e Q_m(d_je) cbar_e ----
static double cbar_of(int64_t l) { return std::sin(1.3 * (double)l) + 0.1; }

struct Moments {
    float f0h = 0.f, f0l = 0.f, f1h = 0.f, f1l = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f, f5 = 0.f, f6 = 0.f, f7 = 0.f;
};

// out[m] += sum_r a_{iv,m,r} F_r, m >= 1 of the interval (the kernel's rs_flush)
static void flush_T(const RangeTables& rt, int iv, const Moments& F, double* out) {
    const int m0 = std::max(1, rt.mr[2 * iv]), m1 = rt.mr[2 * iv + 1];
    for (int m = m0; m <= m1; m++) {
        const float* c = &rt.coef[((size_t)iv * rt.nm + m) * 12];
        float h = 0.f, l = 0.f;
        rs::acc_mac(h, l, c[0], c[1], F.f0h, F.f0l);
        rs::acc_mac(h, l, c[2], c[3], F.f1h, F.f1l);
        float r = rs::fma_(c[5], F.f2, rs::fma_(c[4], F.f2, 0.f));
        r = rs::fma_(c[7], F.f3, rs::fma_(c[6], F.f3, r));
        r = rs::fma_(c[8], F.f4, r);
        r = rs::fma_(c[9], F.f5, r);
        r = rs::fma_(c[10], F.f6, r);
        r = rs::fma_(c[11], F.f7, r);
        rs::acc_add(h, l, r, 0.f);
        out[m] += (double)h + (double)l;
    }
}

// F += cbar z^r (the kernel's rs_moments_add)
static void moments_add(Moments& F, float zh, float zl, float ch, float cl) {
    rs::acc_add(F.f0h, F.f0l, ch, cl);
    rs::acc_mac(F.f1h, F.f1l, zh, zl, ch, cl);
    const float z2 = rs::mul(zh, zh);
    float p = rs::mul(z2, ch);
    F.f2 = rs::add(F.f2, p);
    p = rs::mul(p, zh);
    F.f3 = rs::add(F.f3, p);
    p = rs::mul(p, zh);
    F.f4 = rs::add(F.f4, p);
    p = rs::mul(p, zh);
    F.f5 = rs::add(F.f5, p);
    p = rs::mul(p, zh);
    F.f6 = rs::add(F.f6, p);
    p = rs::mul(p, zh);
    F.f7 = rs::add(F.f7, p);
}

// one output block of 128 springs, traversed as k_rs_local_T does: the forward block's window in
// chunks of 32 inputs, each output walking its inputs side by side and flushing the moments of its
// current interval when the interval changes
static void block_sums_T(const HostPlan& hp, int64_t B, std::vector<double>& out) {
    const RangeTables& rt = hp.rt;
    const int64_t M = hp.P.M, j0 = B * kRsTTargets;
    const int nT = (int)std::min<int64_t>(kRsTTargets, M - j0);
    const int64_t b = j0 / kRsTargets;
    const int wlo = hp.blk_win[4 * b], inlo = hp.blk_win[4 * b + 1], inhi = hp.blk_win[4 * b + 2],
              whi = hp.blk_win[4 * b + 3];
    const int nL = std::max(0, inhi - wlo), total = nL + std::max(0, whi - inlo);
    const double xa = hp.x[j0], span = hp.x[j0 + nT - 1] - xa;
    const rs::Grid G = rs::grid_of(span, hp.P.delta);
    std::vector<float> ivt(4 * (size_t)rt.nint);
    for (int iv = 0; iv < rt.nint; iv++) rs::interval_on_grid(rt.mid[iv], rt.ih[iv], G, &ivt[4 * (size_t)iv]);
    for (int t = 0; t < nT; t++) {
        const int64_t j = j0 + t;
        float hj, lj;
        rs::grid_split(hp.x[j] - xa, G, hj, lj);
        int64_t lbj = j;
        while (lbj > 0 && hp.x[lbj - 1] == hp.x[j]) lbj--;
        rs::Track trL, trR;
        rs::track_to(ivt.data(), 0, hj, lj, trL);
        rs::track_to(ivt.data(), 0, -hj, -lj, trR);
        int cur = -1;
        Moments F;
        double* o = &out[(size_t)j * rt.nm];
        const int nbl = hp.nb_lo[j], nbc = hp.nb_cnt[j];
        for (int v = 0; v < total; v++) {
            const bool left = v < nL;
            const int e = left ? wlo + v : inlo + (v - nL);
            const double xr = xext(hp, e) - xa;
            float h, l;
            rs::grid_split(xr, G, h, l);
            const int lohi = rs::source_range(xr, left, span, hp.P.delta, hp.P.dt, rt.bp2.data(), rt.cell.data(),
                                              rt.cell_scale, rt.nint);
            if ((lohi & 0x7fff) > (lohi >> 16) || (left ? e >= lbj : e < lbj)) continue;
            float zh, zl;
            rs::Track& tr = left ? trL : trR;
            const float bh = left ? hj : -hj, bl = left ? lj : -lj;
            if (left) {
                rs::z_of<-1>(tr, h, l, zh, zl);
                if (std::fabs(zh) > rs::kZTol)
                    rs::walk<-1>(ivt.data(), rt.cell.data(), rt.cell_scale, rt.nint, bh, bl, h, l, tr, zh, zl);
                if (lohi & 0x8000)
                    rs::near_side<-1>(ivt.data(), rt.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, h, l, tr, zh, zl);
            } else {
                rs::z_of<1>(tr, h, l, zh, zl);
                if (std::fabs(zh) > rs::kZTol)
                    rs::walk<1>(ivt.data(), rt.cell.data(), rt.cell_scale, rt.nint, bh, bl, h, l, tr, zh, zl);
                if (lohi & 0x8000)
                    rs::near_side<1>(ivt.data(), rt.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, h, l, tr, zh, zl);
            }
            if (!(std::fabs(zh) <= rs::kZTol)) continue;
            if (tr.iv != cur) {
                if (cur >= 0) flush_T(rt, cur, F, o);
                cur = tr.iv;
                F = Moments();
            }
            const double c = cbar_of(e < 0 ? e + M : (e >= M ? e - M : e));
            const float ch = (float)c;
            moments_add(F, zh, zl, ch, (float)(c - (double)ch));
        }
        if (cur >= 0) flush_T(rt, cur, F, o);
    }
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
    if (std::strcmp(mode, "tsum") == 0) {
        // the transposed sums per m against the stored FP64 weights: ref_j[m] = sum_e Q_m(d_je) cbar_e
        const int nm = hr.rt.nm;
        std::vector<double> tref((size_t)M * nm, 0.0), tgot((size_t)M * nm, 0.0);
        const LocalCSR& C = hs.loc;
        for (int64_t j = 0; j < M; j++)
            for (int64_t e = C.row_ptr[j]; e < C.row_ptr[j + 1]; e++) {
                const int lo = C.mrange[e] & 0xffff, cnt = C.mrange[e] >> 16;
                for (int c = 0; c < cnt; c++) tref[(size_t)j * nm + lo + c] += C.w[C.woff[e] + c] * cbar_of(C.src[e]);
            }
        const int64_t nb = (M + kRsTTargets - 1) / kRsTTargets;
        for (int64_t B = 0; B < nb; B++) block_sums_T(hr, B, tgot);
        double worst = 0.0, scale = 0.0;
        for (size_t i = 0; i < tref.size(); i++) {
            worst = std::max(worst, std::fabs(tgot[i] - tref[i]));
            scale = std::max(scale, std::fabs(tref[i]));
        }
        std::printf("ok %.3e %zu\n", worst / scale, C.src.size());
        return 0;
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
