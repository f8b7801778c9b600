// Bodies of the reverse-time (adjoint) step of the discrete scheme, one output element each,
// written for both the GPU kernels (adjoint.cu) and a host check that runs them over the same
// tables.  Complex values are interleaved (re, im) doubles.
//
// The forward step n -> n+1 is linear in the state (sigma ring, S ring, alpha, alpha') and the
// forcing, so the gradient of a loss of the receiver fields follows from the transposed pieces
// taken in reverse order (real inner product Re <a, b>):
//   receivers  u_r = 1/2 (sum_{m>=1} Q_m sigma^{n+1-m} + sum_{d<dt} Q_0 sigma^{n+1}) + u_H(x_r)
//              -> sigmabar^{n+1-m}[src] += 1/2 Q_m ubar_r,  alphabar_k += w_k e^{i k x_r} ubar_r
//   solve      (I + S) sigma^{n+1} = rhs (eq. linearSystem)  ->  rhsbar = (I + S)^{-T} sigmabar
//   local sum  c_j = sum_{m>=1} Q_m sigma_src^{n+1-m} (Sec. 4.1)  ->  sigmabar += Q_m cbar_j
//   type-2     u_H = sum_{|k|<=K} alpha_k e^{-i k x}  ->  alphabar_k += w_k 2 pi S_k[u_Hbar]
//   projection (Sec. 4.4) -> its transpose (below)
//   modes      alpha^{n+1} = cos alpha + sin/k alpha' + h, alpha'^{n+1} = -k sin alpha + cos alpha'
//              + g, h = sum_m dt p_k(m dt) S^{n-m}, g likewise with q_k (eqs.
//              alphakEvolutionFormulas, hkcompdisc)  ->  the transposed rotation and FIR
//   type-1     S_k = (1/2 pi) sum_j sigma_j e^{i k x_j} (eq. densco)
//              -> sigmabar_j += (1/2 pi) Re sum_{k=0}^{K} e^{-i k x_j} Sbar_k
// with w_0 = 1, w_k = 2 (k >= 1).  The stiffness enters through rhs = -beta f - beta/2 c - beta u_H
// and S = diag(beta/2) Q_0; since sigma_j + beta_j/2 (Q_0 sigma)_j = rhs_j, the derivative of the
// step's residual with respect to beta_j reduces to sigma_j^{n+1} / beta_j, and
//   dL/dbeta_j = sum_n rhsbar_j^n sigma_j^{n+1} / beta_j.
#pragma once

#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define WAVE1D_HD __host__ __device__ __forceinline__
#else
#define WAVE1D_HD inline
#endif

namespace wave1d {
namespace adj {

// FP32 operations rounded to nearest without contraction or reassociation (rounding intrinsics on
// the GPU; on the host, ISO C++ float arithmetic, which compilers do not contract by default)
#ifdef __CUDA_ARCH__
WAVE1D_HD float f_add(float a, float b) { return __fadd_rn(a, b); }
WAVE1D_HD float f_sub(float a, float b) { return __fsub_rn(a, b); }
WAVE1D_HD float f_mul(float a, float b) { return __fmul_rn(a, b); }
WAVE1D_HD float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
WAVE1D_HD float f_add(float a, float b) { return a + b; }
WAVE1D_HD float f_sub(float a, float b) { return a - b; }
WAVE1D_HD float f_mul(float a, float b) { return a * b; }
WAVE1D_HD float f_fma(float a, float b, float c) { return std::fma(a, b, c); }
#endif

// Compensated FP32 pairs: a value is hi + lo with |lo| <= ulp(hi)/2.  (sh, sl) += (wh + wl)(vh + vl)
// with the product's rounding error recovered by fused multiply-adds and the sum's by a two-sum
// (Knuth), dropping wl vl (relative 2^-48): the arithmetic of the forward local sum.
WAVE1D_HD void pair_mac(float& sh, float& sl, float wh, float wl, float vh, float vl) {
    const float p = f_mul(wh, vh);
    float e = f_fma(wh, vh, -p);
    e = f_fma(wh, vl, e);
    e = f_fma(wl, vh, e);
    const float s = f_add(sh, p);
    const float bb = f_sub(s, sh);
    const float t = f_add(f_sub(sh, f_sub(s, bb)), f_sub(p, bb));
    sh = s;
    sl = f_add(sl, f_add(t, e));
}

// slot of time index q in a ring of `ring` slots (q may be negative)
WAVE1D_HD int slot(int64_t q, int ring) {
    int64_t r = q % ring;
    return (int)(r < 0 ? r + ring : r);
}

// One lane of a local-sum item of row l, read in the transposed direction.  The LocalItems
// layout: lane `lane` holds source rank 32 c + lane of the row, slice t of the item is
// m = mfirst + s0 + t, and the weight of slice t is the (hi, lo) float pair at weight index
// wbase + 64 (t / 2) + 2 lane + (t % 2).  Q_m(d) depends on the pair only through its distance,
// so row l's weight for source j is row j's weight for source l, and the transposed local sum
// at l is
//   sigmabar^{q - m}[l] += sum_{j in row l} Q_m(d_lj) cbar_j .
// The lane adds Q_m (cbh + cbl) (cbar of its source as an FP32 pair) into the pair accumulator
// acc(m) for every slice with a non-zero weight; its caller owns the sums of row l, so no two
// writers meet.
template <class Acc>
WAVE1D_HD void item_lane_gather(const float* w, int64_t wbase, int s0, int len, int lane, int mfirst,
                                float cbh, float cbl, Acc acc) {
    for (int t = 0; t < len; t++) {
        const float* e = w + 2 * (wbase + 64 * (int64_t)(t >> 1) + 2 * lane + (t & 1));
        if (e[0] != 0.0f) {
            float* a = acc(mfirst + s0 + t);
            pair_mac(a[0], a[1], e[0], e[1], cbh, cbl);
        }
    }
}

// an FP64 value as an FP32 pair (hi = fl(v), lo = fl(v - hi))
WAVE1D_HD void split_pair(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// The receivers' transposed readout at source l, from the receiver weights regrouped by source
// (ReceiverColumns: entries [ptr[l], ptr[l + 1]), receiver rcv[e], m range mrange[e] = m_lo |
// count << 16, weights w[woff[e] ..]):
//   sigmabar^{q - m}[l] += 1/2 Q_m(d_rl) ubar_r   for m >= 0, delivered as add(ring slot, value).
template <class Add>
WAVE1D_HD void receivers_T_source(int64_t l, const int64_t* ptr, const int32_t* rcv, const int32_t* mrange,
                                  const int64_t* woff, const double* w, const double* ubar, int64_t q,
                                  int ring, Add add) {
    for (int64_t e = ptr[l]; e < ptr[l + 1]; e++) {
        const double coef = 0.5 * ubar[rcv[e]];
        if (coef == 0.0) continue;
        const int mlo = mrange[e] & 0xffff, cnt = mrange[e] >> 16;
        for (int c = 0; c < cnt; c++) add(slot(q - mlo - c, ring), w[woff[e] + c] * coef);
    }
}

// Transposed block solve for member l of a block of s members (members m0 .. m0 + s - 1 of
// blk_members, inverse stored column-major: invT[l s + i] = inverse[i][l]):
//   rhsbar[member l] = sum_i inverse[i][l] sigbar[member i]
WAVE1D_HD double solve_T(const double* invT, const int32_t* members, int64_t m0, int s, int l,
                         const double* sigbar) {
    double a0 = 0.0, a1 = 0.0;
    const double* col = invT + (int64_t)l * s;
    int i = 0;
    for (; i + 1 < s; i += 2) {
        a0 = fma(col[i], sigbar[members[m0 + i]], a0);
        a1 = fma(col[i + 1], sigbar[members[m0 + i + 1]], a1);
    }
    if (i < s) a0 = fma(col[i], sigbar[members[m0 + i]], a0);
    return a0 + a1;
}

// alphabar_k += w_k (2 pi S1_k + sum_r ubar_r e^{i k x_r}): the adjoints of the springs' u_H
// (S1 = type-1 of u_Hbar) and of the receivers' u_H, on alpha^{n+1} after its projection.
WAVE1D_HD void modes_in(int k, const double* S1, const double* xr, const double* ubar, int64_t R,
                        double* ab) {
    const double two_pi = 6.283185307179586476925286766559;
    const double wk = k == 0 ? 1.0 : 2.0;
    double re = two_pi * S1[2 * k], im = two_pi * S1[2 * k + 1];
    for (int64_t r = 0; r < R; r++) {
        const double a = (double)k * xr[r];
        re = fma(ubar[r], cos(a), re);
        im = fma(ubar[r], sin(a), im);
    }
    ab[2 * k] = fma(wk, re, ab[2 * k]);
    ab[2 * k + 1] = fma(wk, im, ab[2 * k + 1]);
}

// Transposed projection (Sec. 4.4), grid part, at rolled-off point pt of the 2K-point grid
// (index ig, x = ig pi / K, tw2K[a] = e^{i pi a / K}).  The forward projection changes the grid
// values u, v of the field (modes |k| <= K-1) by du = (phi - 1) u, dv = phi' u + (phi - 1) v and
// adds (1/2K) sum du e^{i k x} to alpha_k (k < K).  Its adjoint at the point:
//   Du = (1/2K) sum_{k<K} Re(alphabar_k e^{-i k x}),  Dv likewise from alpha'bar,
//   ubar = (phi - 1) Du + phi' Dv,  vbar = (phi - 1) Dv.
WAVE1D_HD void rbc_grid_T(int ig, int K, const double* tw2K, const double* ab, const double* apb,
                          double phi, double dphi, double* ubar, double* vbar) {
    const int64_t twoK = 2 * (int64_t)K;
    double su = ab[0], sv = apb[0];
    for (int k = 1; k < K; k++) {
        const int64_t a = ((int64_t)k * ig) % twoK;
        const double c = tw2K[2 * a], s = tw2K[2 * a + 1];          // e^{+i k x}
        su += ab[2 * k] * c + ab[2 * k + 1] * s;                     // Re(ab e^{-i k x})
        sv += apb[2 * k] * c + apb[2 * k + 1] * s;
    }
    const double inv = 1.0 / (double)twoK;
    const double Du = su * inv, Dv = sv * inv;
    *ubar = fma(phi - 1.0, Du, dphi * Dv);
    *vbar = (phi - 1.0) * Dv;
}

// Transposed projection, mode part: the identity on k < K plus the grid values' dependence on
// alpha (u = Re alpha_0 + 2 sum_{k=1}^{K-1} Re(alpha_k e^{-i k x})); alpha_K does not reach the
// projected field, whose alpha_K is zero, so its adjoint is zero.
WAVE1D_HD void rbc_update_T(int k, int K, int npts, const int32_t* idx, const double* tw2K,
                            const double* uvbar, double* ab, double* apb) {
    if (k == K) {
        ab[2 * k] = ab[2 * k + 1] = 0.0;
        apb[2 * k] = apb[2 * k + 1] = 0.0;
        return;
    }
    const int64_t twoK = 2 * (int64_t)K;
    double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
    for (int pt = 0; pt < npts; pt++) {
        const int64_t a = ((int64_t)k * idx[pt]) % twoK;
        const double c = tw2K[2 * a], s = tw2K[2 * a + 1];
        const double u = uvbar[2 * pt], v = uvbar[2 * pt + 1];
        ur = fma(u, c, ur);
        ui = fma(u, s, ui);
        vr = fma(v, c, vr);
        vi = fma(v, s, vi);
    }
    if (k == 0) {                        // Re alpha_0 only
        ab[0] += ur;
        apb[0] += vr;
    } else {
        ab[2 * k] = fma(2.0, ur, ab[2 * k]);
        ab[2 * k + 1] = fma(2.0, ui, ab[2 * k + 1]);
        apb[2 * k] = fma(2.0, vr, apb[2 * k]);
        apb[2 * k + 1] = fma(2.0, vi, apb[2 * k + 1]);
    }
}

// Transposed mode update of step n for mode k (K1 = K + 1 modes):
//   (hbar, gbar) = (alphabar_k, alpha'bar_k) of alpha^{n+1};
//   alphabar_k <- cos hbar - k sin gbar,  alpha'bar_k <- (sin/k) hbar + cos gbar   (alpha^n);
//   Sbar^{n-m}_k += dt p_k(m dt) hbar + dt q_k(m dt) gbar,  m = 0 .. W-1  (ring of W slots);
// then Sbar^n_k is complete: it is taken out of the ring (its slot zeroed for S^{n-W}) and turned
// into the type-2 input a2_k = Sbar^n_k / (2 pi w_k) whose evaluation at the springs is
// sigmabar^n; the imaginary part of mode 0 is dropped (S_0 is real).
WAVE1D_HD void modes_T(int k, int K1, int W, int64_t n, const double* rot, const double* pq,
                       double* ab, double* apb, double* Sb, double* a2) {
    const double hr = ab[2 * k], hi = ab[2 * k + 1], gr = apb[2 * k], gi = apb[2 * k + 1];
    const double cs = rot[3 * k], so = rot[3 * k + 1], ks = rot[3 * k + 2];
    ab[2 * k] = fma(cs, hr, -ks * gr);
    ab[2 * k + 1] = fma(cs, hi, -ks * gi);
    apb[2 * k] = fma(so, hr, cs * gr);
    apb[2 * k + 1] = fma(so, hi, cs * gi);
    for (int m = 0; m < W; m++) {
        const double wp = pq[2 * ((int64_t)m * K1 + k)], wq = pq[2 * ((int64_t)m * K1 + k) + 1];
        double* s = Sb + 2 * ((int64_t)slot(n - m, W) * K1 + k);
        s[0] = fma(wp, hr, fma(wq, gr, s[0]));
        s[1] = fma(wp, hi, fma(wq, gi, s[1]));
    }
    double* s = Sb + 2 * ((int64_t)slot(n, W) * K1 + k);
    const double scale = (k == 0 ? 1.0 : 0.5) / 6.283185307179586476925286766559;
    a2[2 * k] = s[0] * scale;
    a2[2 * k + 1] = k == 0 ? 0.0 : s[1] * scale;
    s[0] = s[1] = 0.0;
}

}  // namespace adj
}  // namespace wave1d
