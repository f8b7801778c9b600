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
// r >= 2 (below 2 % of max |Q|) are single floats.  Positions are split on a grid of the target
// block (below), so that d - mid_iv is one exact FP32 difference plus a small rounded part, and z
// carries about 3e-11 absolute error.
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

// four consecutive floats from a 16-byte aligned address (one vector load on the device)
struct F4 {
    float x, y, z, w;
};
WAVE1D_RS_HD F4 load4(const float* p) {
#ifdef __CUDA_ARCH__
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
#else
    return {p[0], p[1], p[2], p[3]};
#endif
}

// acc += e0 + z (e1 + z P(z)),  P(z) = e2 + z (e3 + z (e4 + z (e5 + z (e6 + z e7)))),
// z = zh + zl normalised; r0 = (e0h e0l e1h e1l), r1 = (e2 .. e5), r2 = (e6 e7 - -)
WAVE1D_RS_HD void evec_eval4(const F4& r0, const F4& r1, const F4& r2, float zh, float zl, float& ah, float& al) {
    float P = fma_(r2.y, zh, r2.x);                 // e7 z + e6
    P = fma_(P, zh, r1.w);                          // + e5
    P = fma_(P, zh, r1.z);
    P = fma_(P, zh, r1.y);
    P = fma_(P, zh, r1.x);                          // P(z)
    // w = e1 + z P as a pair
    float wh, we;
    two_sum(r0.z, mul(zh, P), wh, we);
    const float wl = add(r0.w, we);
    // z w as a pair (p, pe)
    const float p = mul(zh, wh);
    float pe = fma_(zh, wh, -p);
    pe = fma_(zh, wl, pe);
    pe = fma_(zl, wh, pe);
    // acc += e0 + z w
    float s, se;
    two_sum(r0.x, p, s, se);
    acc_add(ah, al, s, add(r0.y, add(pe, se)));
}

// the same from a packed record e (12 floats, 16-byte aligned)
WAVE1D_RS_HD void evec_eval(const float* e, float zh, float zl, float& ah, float& al) {
    evec_eval4(load4(e), load4(e + 4), load4(e + 8), zh, zl, ah, al);
}

// the same from an e-vector held in registers
WAVE1D_RS_HD void evec_eval_v(const EVec& v, float zh, float zl, float& ah, float& al) {
    evec_eval4(F4{v.e0h, v.e0l, v.e1h, v.e1l}, F4{v.e2, v.e3, v.e4, v.e5}, F4{v.e6, v.e7, 0.f, 0.f}, zh, zl, ah, al);
}

// ---------------------------------------------------------------------------------------------
// Distances on the grid of a target block.  The targets x_a .. x_b of a block and their sources
// lie within span + delta of x_a (span = x_b - x_a), so positions relative to x_a are split as
// x - x_a = h + l, h a multiple of the grid step g = 2^(k - 24) with 2^k > 4 (span + delta) and
// l = fl(x - x_a - h), |l| <= g / 2; interval midpoints the same way.  Sums and differences of two
// such h stay below 2^24 g, so they are exact in FP32: for a source (h, l) and the tracked
// interval's Y = b - mid (b = target for left sources, minus the target for right ones)
//   z = (d - mid) ih = (Y_h -/+ h) ih + (Y_l -/+ l) ih,
// the first product exact through its FMA residual, the second rounded (|Y_l -/+ l| <= 1.5 g).
// ---------------------------------------------------------------------------------------------
struct Grid {
    double g, ig;
};

WAVE1D_RS_HD Grid grid_of(double span, double delta) {
    int k;
    (void)frexp(4.0 * (span + delta), &k);          // 4 (span + delta) < 2^k
    return {ldexp(1.0, k - 24), ldexp(1.0, 24 - k)};
}

// v = h + l on the grid (|v| < 2^k: h is an integer multiple of g below 2^24 g, exact in FP32)
WAVE1D_RS_HD void grid_split(double v, Grid G, float& h, float& l) {
    const double hd = rint(v * G.ig) * G.g;
    h = (float)hd;
    l = (float)(v - hd);
}

// an interval on the block grid: (mid_h, mid_l, ih, 0)
WAVE1D_RS_HD void interval_on_grid(double mid, float ih, Grid G, float* out4) {
    grid_split(mid, G, out4[0], out4[1]);
    out4[2] = ih;
    out4[3] = 0.f;
}

// |z| above which a distance lies outside the tracked interval (z carries about 3e-11; the slack
// lets the walk end where rounding puts a distance on a breakpoint)
constexpr float kZTol = 1.000001f;
// margin of the interval ranges of a source, relative to delta: it covers the FP32 rounding of the
// ranges' end distances and the walk's slack, so every pair's interval lies inside its source's range
constexpr double kRangeMargin = 4e-7;

// Tracked interval of one side (left or right sources) for one target: iv, Y = b - mid_iv, ih_iv.
struct Track {
    int iv;
    float Yh, Yl, ih;
};

// ivt: the block's interval table, 4 floats per interval (interval_on_grid)
WAVE1D_RS_HD void track_to(const float* ivt, int iv, float bh, float bl, Track& t) {
    const F4 v = load4(ivt + 4 * iv);
    t.iv = iv;
    t.Yh = sub(bh, v.x);
    t.Yl = sub(bl, v.y);
    t.ih = v.z;
}

// z = zh + zl (normalised) of the source (h, l) on side S (-1: left sources, d = x_j - x; +1:
// right sources, d = x - x_j) against the tracked interval.  The rounded part (Y_l -/+ l) ih
// reaches about 1e-3, so the two parts are renormalised: the curvature terms of the polynomial
// take zh alone.
template <int S>
WAVE1D_RS_HD void z_of(const Track& t, float h, float l, float& zh, float& zl) {
    const float A = S < 0 ? sub(t.Yh, h) : add(t.Yh, h);    // exact
    const float B = S < 0 ? sub(t.Yl, l) : add(t.Yl, l);
    const float p = mul(A, t.ih);
    two_sum(p, fma_(B, t.ih, fma_(A, t.ih, -p)), zh, zl);
}

// Move the tracked interval to the source's distance: searched afresh through the cell table when
// far off (|z| > 4), then walked in one direction only until |zh| <= kZTol (one direction, so the
// walk ends even where rounding leaves z just outside two neighbouring intervals) or the end of
// [0, delta) is reached (the caller then finds |zh| > kZTol: the pair lies beyond delta).
// cell: kRsCells entries, the interval of the left end of each cell of [0, delta), cell of d =
// floor(d cscale).
template <int S>
WAVE1D_RS_HD void walk(const float* ivt, const int* cell, float cscale, int nint, float bh, float bl, float h, float l,
                       Track& t, float& zh, float& zl) {
    if ((zh > 4.f || zh < -4.f) && !(zh > 0.f && t.iv == nint - 1)) {
        const float dh = S < 0 ? sub(bh, h) : add(bh, h);
        const float d = add(dh, S < 0 ? sub(bl, l) : add(bl, l));
        int c = (int)mul(d, cscale);
        c = c < 0 ? 0 : (c >= kRsCells ? kRsCells - 1 : c);
        track_to(ivt, cell[c], bh, bl, t);
        z_of<S>(t, h, l, zh, zl);
    }
    int dir = 0;
    while (zh > kZTol || zh < -kZTol) {
        const int want = zh > 0.f ? 1 : -1;
        if (dir != 0 && want != dir) break;
        const int nv = t.iv + want;
        if (nv < 0 || nv >= nint) break;
        dir = want;
        track_to(ivt, nv, bh, bl, t);
        z_of<S>(t, h, l, zh, zl);
    }
}

// interval of a float distance: the cell table, then the breakpoints' high parts (bp2 pairs)
WAVE1D_RS_HD int locate_f(const float* bp2, const int* cell, float cscale, int nint, float d) {
    int c = (int)mul(d, cscale);
    c = c < 0 ? 0 : (c >= kRsCells ? kRsCells - 1 : c);
    int iv = cell[c];
    while (iv > 0 && d < bp2[2 * iv]) iv--;
    while (iv + 1 < nint && !(d < bp2[2 * iv + 2])) iv++;
    return iv;
}

// Interval range [lo, hi] of a source's distances to the block's targets (xr = x_e - x_a; left:
// d = x_j - x_e, right: d = x_e - x_j, x_j in [x_a, x_a + span]), lo > hi where none is below
// delta, and whether some distance may lie within rounding of dt (near = 1).  Packed as
// lo | near << 15 | hi << 16 (intervals below 2^15).
WAVE1D_RS_HD int source_range(double xr, bool left, double span, double delta, double dt, const float* bp2,
                              const int* cell, float cscale, int nint) {
    const double marg = kRangeMargin * delta;
    const double dmin = left ? -xr : xr - span, dmax = left ? span - xr : xr;
    if (dmax < 0.0 || !(dmin - marg < delta)) return 1;
    const double d0 = dmin - marg;
    const int lo = locate_f(bp2, cell, cscale, nint, (float)(d0 > 0.0 ? d0 : 0.0));
    const int hi = locate_f(bp2, cell, cscale, nint, (float)(dmax + marg));
    const int near = dmin - marg < dt && dt < dmax + marg ? 1 : 0;
    return lo | near << 15 | hi << 16;
}

// The rule of the implicit part: a pair is near when |x_e - x_j| < dt in FP64 (the spring's window
// of sources), and Q_m, m >= 1, of near pairs comes from the intervals below dt, of the others from
// those at or above it (the interpolation stencils of the two cases differ, so Q_m jumps at
// d = dt).  Where the walk ended on the other side of dt (the distance within rounding of dt), the
// pair moves to the interval next to dt on its side.
template <int S>
WAVE1D_RS_HD void near_side(const float* ivt, int iv_dt, bool near, float bh, float bl, float h, float l, Track& t,
                            float& zh, float& zl) {
    if (near != (t.iv < iv_dt)) {
        track_to(ivt, near ? iv_dt - 1 : iv_dt, bh, bl, t);
        z_of<S>(t, h, l, zh, zl);
    }
}

}  // namespace rs
}  // namespace wave1d
