// Arithmetic of the local sum computed from sorted neighbour ranges (plans opened with
// opts.local_weights = 1), shared by the kernels (range.cu) and host checks.
//
// The local explicit sum of Sec. 4.1 for target j is
//   c_j = sum_l sum_{m >= 1} Q_m(d_jl) sigma_l^{n+1-m},   d_jl = dist(x_j, x_l) < delta.
// Q_m(d) is smooth in d between the breakpoints of the Gauss-Legendre rule (a node crossing a
// multiple of dt, and d = dt), so on interval iv each Q_m is a polynomial of degree 7 in
// z = (d - mid_iv) ih_iv, written a_{iv,m,0} + a_{iv,m,1} z + ... + a_{iv,m,7} z^7.  Per source l
// and interval iv the step's densities fold into one vector
//   e_{l,iv,r} = sum_m a_{iv,m,r} sigma_l^{n+1-m},     r = 0..7,
// and every pair (j, l) with d_jl in interval iv then costs one polynomial in z:
//   sum_m Q_m(d_jl) sigma_l^{n+1-m} = sum_r e_{l,iv,r} z^r.
// Many targets share (l, iv) where springs are dense, so the fold is paid once for all of them.
//
// Precision.  Values are compensated FP32 pairs hi + lo (error-free two-sum and FMA residuals,
// about 48 significant bits); GB300 issues FP32 61 times faster than FP64.  The terms that carry
// the magnitude (r = 0, 1: the interval mean and slope) are pairs throughout; the curvature terms
// r >= 2 (below 2 % of max |Q|) are single floats.  Positions are pairs (x = hi + lo exactly to
// about 1e-14), so pair distances and z keep about 1e-14 absolute.
//
// Every operation is written with round-to-nearest intrinsics on the device, and plainly on the
// host (host checks compile with -ffp-contract=off), so both give the same bits.
#pragma once

#include <cmath>
#include <cstdint>

#include "internal.h"

#ifdef __CUDACC__
#define WAVE1D_RS_HD __host__ __device__ __forceinline__
#else
#define WAVE1D_RS_HD inline
#endif

namespace wave1d {
namespace rs {

struct Pair {
    float hi, lo;
};

WAVE1D_RS_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
WAVE1D_RS_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
WAVE1D_RS_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
WAVE1D_RS_HD float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (Knuth's two-sum, no condition on the operands)
WAVE1D_RS_HD void two_sum(float a, float b, float& s, float& e) {
    s = add(a, b);
    const float bb = sub(s, a);
    e = add(sub(a, sub(s, bb)), sub(b, bb));
}

// (h, l) + (bh, bl) into a normalised pair
WAVE1D_RS_HD Pair pair_add(Pair a, Pair b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = add(e, add(a.lo, b.lo));
    float h, l;
    two_sum(s, e, h, l);
    return {h, l};
}

WAVE1D_RS_HD Pair pair_sub(Pair a, Pair b) { return pair_add(a, Pair{-b.hi, -b.lo}); }

// a < b for normalised pairs
WAVE1D_RS_HD bool pair_lt(Pair a, Pair b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// z = (a - b) s as a pair (zh, zl) with |zl| within a couple of ulp of zh: the difference through
// two-sum and renormalised (the high parts of nearby positions cancel, so the difference's low
// part can be as large as its high part), the product through its FMA residual (a, b normalised
// pairs, s a float scale)
WAVE1D_RS_HD void scaled_diff(Pair a, Pair b, float s, float& zh, float& zl) {
    float d, e;
    two_sum(a.hi, -b.hi, d, e);
    float th, tl;
    two_sum(d, add(e, sub(a.lo, b.lo)), th, tl);
    zh = mul(th, s);
    zl = fma_(tl, s, fma_(th, s, -zh));
}

// acc += (vh + vl), acc kept as an unnormalised pair (hi carries the sum, lo the residuals)
WAVE1D_RS_HD void acc_add(float& ah, float& al, float vh, float vl) {
    float s, e;
    two_sum(ah, vh, s, e);
    ah = s;
    al = add(al, add(vl, e));
}

// acc += (wh + wl)(vh + vl), dropping wl vl (relative 2^-48)
WAVE1D_RS_HD void acc_mac(float& ah, float& al, float wh, float wl, float vh, float vl) {
    const float p = mul(wh, vh);
    float e = fma_(wh, vh, -p);
    e = fma_(wh, vl, e);
    e = fma_(wl, vh, e);
    acc_add(ah, al, p, e);
}

// the pair of a double: hi = fl(v), lo = fl(v - hi)
WAVE1D_RS_HD Pair split(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// ---------------------------------------------------------------------------------------------
// Per-source, per-interval vector e_r (r = 0..7): e0, e1 as pairs, e2..e7 single.
// Coefficient layout per (interval, m): three float4, (a0h, a0l, a1h, a1l), (a2h, a2l, a3h, a3l),
// (a4, a5, a6, a7).  The coefficients a2 and a3 reach a few per cent of max |Q| on the intervals
// just above d = 0 and d = dt, so single floats would move every weight of those intervals by up
// to 5e-10 of max |Q| alike (a systematic change of the scheme); as pairs they are exact to
// 2^-48, and what remains is the rounding of each source's own sums, which differs from source to
// source and averages out in the local sum.
// ---------------------------------------------------------------------------------------------
struct EVec {
    float e0h, e0l, e1h, e1l, e2, e3, e4, e5, e6, e7;
};

WAVE1D_RS_HD void evec_zero(EVec& v) {
    v.e0h = v.e0l = v.e1h = v.e1l = 0.f;
    v.e2 = v.e3 = v.e4 = v.e5 = v.e6 = v.e7 = 0.f;
}

// v += a_{.,m,.} sigma for one m; c01 = (a0h, a0l, a1h, a1l), c23 = (a2h, a2l, a3h, a3l),
// c47 = (a4 .. a7), sigma = (sh, sl)
WAVE1D_RS_HD void evec_mac(EVec& v, const float* c01, const float* c23, const float* c47, float sh, float sl) {
    acc_mac(v.e0h, v.e0l, c01[0], c01[1], sh, sl);
    acc_mac(v.e1h, v.e1l, c01[2], c01[3], sh, sl);
    v.e2 = fma_(c23[1], sh, fma_(c23[0], sh, v.e2));
    v.e3 = fma_(c23[3], sh, fma_(c23[2], sh, v.e3));
    v.e4 = fma_(c47[0], sh, v.e4);
    v.e5 = fma_(c47[1], sh, v.e5);
    v.e6 = fma_(c47[2], sh, v.e6);
    v.e7 = fma_(c47[3], sh, v.e7);
}

// Packed record of an e-vector in shared memory (12 floats: e0h e0l e1h e1l e2..e7, two spare).
constexpr int kERecord = 12;

// acc += e0 + z (e1 + z P(z)),  P(z) = e2 + z (e3 + z (e4 + z (e5 + z (e6 + z e7)))),
// z = zh + zl; e is a packed record
WAVE1D_RS_HD void evec_eval(const float* e, float zh, float zl, float& ah, float& al) {
    float P = fma_(e[9], zh, e[8]);                 // e7 z + e6
    P = fma_(P, zh, e[7]);                          // + e5
    P = fma_(P, zh, e[6]);
    P = fma_(P, zh, e[5]);
    P = fma_(P, zh, e[4]);                          // P(z)
    // w = e1 + z P as a pair
    float wh, we;
    two_sum(e[2], mul(zh, P), wh, we);
    const float wl = add(e[3], we);
    // z w as a pair (p, pe)
    const float p = mul(zh, wh);
    float pe = fma_(zh, wh, -p);
    pe = fma_(zh, wl, pe);
    pe = fma_(zl, wh, pe);
    // acc += e0 + z w
    float s, se;
    two_sum(e[0], p, s, se);
    acc_add(ah, al, s, add(e[1], add(pe, se)));
}

// ---------------------------------------------------------------------------------------------
// Interval of a distance.  bp2: nint + 1 breakpoints as (hi, lo) pairs; tab: kRsCells entries, the
// interval of the left end of each cell of [0, delta), cell of d = floor(d cscale).
// ---------------------------------------------------------------------------------------------
WAVE1D_RS_HD int locate_tab(const float* bp2, const int* tab, float cscale, int nint, Pair d) {
    int c = (int)mul(d.hi, cscale);
    c = c < 0 ? 0 : (c >= kRsCells ? kRsCells - 1 : c);
    int iv = tab[c];
    while (iv > 0 && pair_lt(d, Pair{bp2[2 * iv], bp2[2 * iv + 1]})) iv--;
    while (iv + 1 < nint && !pair_lt(d, Pair{bp2[2 * iv + 2], bp2[2 * iv + 3]})) iv++;
    return iv;
}

// Tracked interval of one side (left or right sources) for one target: the interval iv of the last
// source's distance and Y = x_j -/+ mid_iv, so z = (Y - x_e) ih (left) or (x_e - Y) ih (right).
struct Track {
    int iv;
    Pair Y;
};

// Interval and z of the pair (target Xj, source X) on side `left`: from the tracked interval, moved
// to the pair's side of dt (near pairs below it, far pairs at or above it), then walked in one
// direction only until z lies in [-1, 1] (to rounding; one direction, so the walk ends even where
// rounding leaves z just outside two neighbouring intervals), or searched afresh when far off.
// mid2 / ih: the intervals' midpoints (pairs) and scales.  Returns false where the pair lies beyond
// delta.
WAVE1D_RS_HD bool pair_z(const float* bp2, const float* mid2, const float* ih, const int* tab, float cscale,
                         int nint, int iv_dt, bool left, bool near, Pair Xj, Pair X, Track& tr, float& zh,
                         float& zl) {
    int iv = tr.iv;
    if (iv >= 0 && (near ? iv >= iv_dt : iv < iv_dt)) iv = near ? iv_dt - 1 : iv_dt;
    if (iv < 0) iv = locate_tab(bp2, tab, cscale, nint, left ? pair_sub(Xj, X) : pair_sub(X, Xj));
    iv = near ? (iv < iv_dt - 1 ? iv : iv_dt - 1) : (iv > iv_dt ? iv : iv_dt);
    if (iv != tr.iv) {
        const Pair mid{mid2[2 * iv], mid2[2 * iv + 1]};
        tr.Y = pair_add(Xj, left ? Pair{-mid.hi, -mid.lo} : mid);
    }
    int dir = 0;
    for (int pass = 0;; pass++) {
        const float sc = ih[iv];
        if (left) scaled_diff(tr.Y, X, sc, zh, zl);
        else scaled_diff(X, tr.Y, sc, zh, zl);
        int nv = iv;
        if (pass == 0 && (zh > 4.f || zh < -4.f)) {
            nv = locate_tab(bp2, tab, cscale, nint, left ? pair_sub(Xj, X) : pair_sub(X, Xj));
            nv = near ? (nv < iv_dt - 1 ? nv : iv_dt - 1) : (nv > iv_dt ? nv : iv_dt);
        } else {
            const int want = zh > 1.000001f ? 1 : (zh < -1.000001f ? -1 : 0);
            if (want == 0 || (dir != 0 && want != dir)) break;
            nv = iv + want;
            if (nv < 0 || nv >= nint || (near ? nv >= iv_dt : nv < iv_dt)) break;
            dir = want;
        }
        if (nv == iv) break;
        iv = nv;
        const Pair mid{mid2[2 * iv], mid2[2 * iv + 1]};
        tr.Y = pair_add(Xj, left ? Pair{-mid.hi, -mid.lo} : mid);
    }
    tr.iv = iv;
    return !(zh > 1.000001f && iv == nint - 1);
}

}  // namespace rs
}  // namespace wave1d
