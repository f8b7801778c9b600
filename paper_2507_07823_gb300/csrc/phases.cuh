// The phases of one WFP time step n -> n+1 as device functions.  The standalone per-stage kernels
// (kernels.cu, history.cu) and the one-launch step kernel (step.cu) are both built from them, so
// the two paths run the same arithmetic.
//
// Every phase works with any block size that is a multiple of 32.  Values another block of the
// same launch may have produced (Y, T, the fine grid, item partials, right-hand sides) are read
// with __ldcg (L2, not the non-coherent L1 path), so the phases stay correct inside one kernel
// whose blocks hand data to each other across a grid-wide barrier.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "internal.h"
#include "../../include/wave1d.h"

namespace wave1d {

// ---------------------------------------------------------------------------------------------
// compensated FP32 pairs: a value is hi + lo with |lo| <= ulp(hi)/2 (error-free transformations,
// written with rounding intrinsics so the compiler neither contracts nor reassociates them)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += (wh + wl) (vh + vl), dropping wl vl (relative 2^-48)
__device__ __forceinline__ void pair_mac(float& sh, float& sl, float2 w, float2 v) {
    float p = __fmul_rn(w.x, v.x);
    float e = __fmaf_rn(w.x, v.x, -p);
    e = __fmaf_rn(w.x, v.y, e);
    e = __fmaf_rn(w.y, v.x, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

__device__ __forceinline__ void pair_add(float& sh, float& sl, float oh, float ol) {
    float s, t;
    two_sum(sh, oh, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(ol, t));
}

__device__ __forceinline__ void pair_warp_sum(float& sh, float& sl) {
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, sh, o);
        float ol = __shfl_xor_sync(0xffffffffu, sl, o);
        pair_add(sh, sl, oh, ol);
    }
}

// ---------------------------------------------------------------------------------------------
// local explicit sum (Sec. 4.1), one work item = 32 sources of one target row (see LocalItems):
//   partial = sum_t sum_lanes Q[slice s0 + t][rank] sigma_src^{n+1-m},  m = m_first + s0 + t
// The density ring sig2 has 2 ring slots (slot s and s + ring hold the same values), so the slot
// of slice s0 + t is b0 - t with b0 in [ring, 2 ring): the walk never wraps.  Each element is one
// contiguous 256-byte weight line per warp, one density load and one compensated multiply-add.
// The ring holds sigma^{<= n} only, written by earlier launches, so the read-only path is safe.
// Weights and source lists are read once per step: they stream through L2 with the evict-first
// policy (ld.global.cs), which keeps the density ring and the history pipeline's few MB of state
// resident in L2 while hundreds of MB of weights pass through it.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void local_item(const float2* __restrict__ sig2, int64_t M, int ring, int q,
                                           int mfirst, int s0, int len, const float4* __restrict__ wp,
                                           int sj, float& sh, float& sl) {
    int b0 = (q - mfirst - s0) % ring;
    if (b0 < 0) b0 += ring;
    b0 += ring;
    const float2* sp = sig2 + (int64_t)b0 * M + sj;
    int t = 0;
    for (; t + 8 <= len; t += 8) {
        float4 w01 = __ldcs(wp + 32 * (t >> 1)), w23 = __ldcs(wp + 32 * ((t >> 1) + 1));
        float4 w45 = __ldcs(wp + 32 * ((t >> 1) + 2)), w67 = __ldcs(wp + 32 * ((t >> 1) + 3));
        float2 v0 = __ldg(sp), v1 = __ldg(sp - M), v2 = __ldg(sp - 2 * M), v3 = __ldg(sp - 3 * M);
        float2 v4 = __ldg(sp - 4 * M), v5 = __ldg(sp - 5 * M), v6 = __ldg(sp - 6 * M), v7 = __ldg(sp - 7 * M);
        pair_mac(sh, sl, make_float2(w01.x, w01.y), v0);
        pair_mac(sh, sl, make_float2(w01.z, w01.w), v1);
        pair_mac(sh, sl, make_float2(w23.x, w23.y), v2);
        pair_mac(sh, sl, make_float2(w23.z, w23.w), v3);
        pair_mac(sh, sl, make_float2(w45.x, w45.y), v4);
        pair_mac(sh, sl, make_float2(w45.z, w45.w), v5);
        pair_mac(sh, sl, make_float2(w67.x, w67.y), v6);
        pair_mac(sh, sl, make_float2(w67.z, w67.w), v7);
        sp -= 8 * M;
    }
    for (; t < len; t += 2) {
        float4 w = __ldcs(wp + 32 * (t >> 1));
        pair_mac(sh, sl, make_float2(w.x, w.y), __ldg(sp));
        pair_mac(sh, sl, make_float2(w.z, w.w), __ldg(sp - M));
        sp -= 2 * M;
    }
}

// One warp per item, items handed out by the atomic counter item_ctr in item_order (spring and
// receiver items together, longest first, so the last items taken are short); the counter is
// reset once every item of the step is done.  Each item's partial sum, one warp reduction of the
// lanes' compensated pairs, goes to l_part / r_part at the item's own index, so the rows sum
// their items' partials later in item order, whatever order the items ran in.
__device__ __forceinline__ void local_items_loop(const DevPlan& P, int64_t n) {
    const int lane = threadIdx.x & 31;
    const int q = ring_slot(n + 1, P.ring);
    const unsigned long long total = (unsigned long long)(P.l_nitems + P.r_nitems);
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(P.item_ctr, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total) break;
        const int64_t o = __ldg(P.item_order + g);
        float sh = 0.f, sl = 0.f;
        if (o < P.l_nitems) {
            const int sj = __ldcs(P.l_src + o * 32 + lane);
            local_item((const float2*)P.sig2, P.M, P.ring, q, P.l_mfirst, __ldg(P.l_s0 + o), __ldg(P.l_len + o),
                       (const float4*)(P.l_w + 2 * __ldg(P.l_wbase + o)) + lane, sj, sh, sl);
            pair_warp_sum(sh, sl);
            if (lane == 0) P.l_part[o] = (double)sh + (double)sl;
        } else {
            const int64_t it = o - P.l_nitems;
            const int sj = __ldcs(P.r_src + it * 32 + lane);
            local_item((const float2*)P.sig2, P.M, P.ring, q, P.r_mfirst, __ldg(P.r_s0 + it), __ldg(P.r_len + it),
                       (const float4*)(P.r_w + 2 * __ldg(P.r_wbase + it)) + lane, sj, sh, sl);
            pair_warp_sum(sh, sl);
            if (lane == 0) P.r_part[it] = (double)sh + (double)sl;
        }
    }
}

// L2 prefetch of [base, base + bytes), one 128-byte line per thread-step, kept with the
// evict-last priority (threads tid = 0 .. nthreads - 1 share the range)
__device__ __forceinline__ void prefetch_l2(const void* base, size_t bytes, int64_t tid, int64_t nthreads) {
    const char* p = (const char*)base;
    for (size_t off = (size_t)tid * 128; off < bytes; off += (size_t)nthreads * 128)
        asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p + off));
}

// ---------------------------------------------------------------------------------------------
// History pipeline (Sec. 3): type-1 NUFFT, mode update, type-2 NUFFT's FFT.  The fine grid of nf
// reals is viewed as L = nf/2 complex points z[r] = G[2r] + i G[2r+1], L = L1 L2, r = i2 + L2 i1
// (column i2), k = k1 + L1 k2 (row k1).
//   cols_phase   spreading of sigma^n into column i2's points (eq. densco), FFT over i1 (sign +),
//                twiddle e^{+2 pi i i2 k1/L}  ->  Y[k1 L2 + i2]
//   rows_phase   rows k1 and L1 - k1 together: FFT over i2 -> Z_k for k = k1 + L1 k2; the modes of
//                the two rows (each needs Z_k and Z_{L-k}, which lie in the pair) are advanced
//                (eqs. hkcompdisc, alphakEvolutionFormulas) and replaced by their type-2 spectrum;
//                then the first pass of the inverse FFT: FFT over k2 (sign -), twiddle
//                e^{-2 pi i k1 i2/L}  ->  T[k1 L2 + i2]
//   icols_phase  FFT over k1 (sign -) of T[k1 L2 + i2]  ->  z'[i2 + L2 i1], i.e. the grid G'.
// ---------------------------------------------------------------------------------------------

// shared memory of the phases (bytes): a line of L1 or two lines of L2 points and the line
// twiddles
__host__ __device__ __forceinline__ size_t cols_phase_smem(int L1) { return (size_t)16 * (L1 + L1 / 2); }
__host__ __device__ __forceinline__ size_t rows_phase_smem(int L2) { return (size_t)16 * (2 * L2 + L2 / 2); }
__host__ __device__ __forceinline__ size_t icols_phase_smem(int L1) { return (size_t)16 * (L1 + L1 / 2); }

// Spreading (eq. densco) into column i2: one thread per real c = 2 i1 + h of the column's points,
// whose entries [g_ptr[c], g_ptr[c + 1]) (rows in column-pass order) are summed with fused
// multiply-adds in entry order, eight loads in flight at a time; then the FFT over i1.
__device__ __forceinline__ void cols_phase(const DevPlan& P, int64_t n, double2* __restrict__ Y, int i2,
                                           unsigned char* smraw) {
    const int L1 = P.L1, L = P.L, bd = blockDim.x, tid = threadIdx.x;
    double2* line = (double2*)smraw;
    double2* twN = line + L1;
    const double* sg = P.sig + (int64_t)ring_slot(n, P.ring) * P.M;
    const int32_t* gp = P.g_ptr + (int64_t)i2 * 2 * L1;
    const double2* tw = (const double2*)P.twiddle;
    const int logL1 = 31 - __clz(L1);
    for (int t = tid; t < L1 / 2; t += bd) twN[t] = __ldg(tw + t * (L / L1));
    const double2 twk = tid < L1 ? __ldg(tw + (((int64_t)i2 * tid) & (L - 1))) : make_double2(0.0, 0.0);
    for (int c = tid; c < 2 * L1; c += bd) {
        int e = __ldg(gp + c);
        const int e1 = __ldg(gp + c + 1);
        double acc = 0.0;
        for (; e < e1; e += 8) {
            int sidx[8];
            double wv[8], v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                sidx[u] = e + u < e1 ? __ldg(P.g_src + e + u) : 0;
                wv[u] = e + u < e1 ? __ldg(P.g_w + e + u) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = __ldg(sg + sidx[u]);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (e + u < e1) acc = fma(wv[u], v[u], acc);
        }
        ((double*)line)[2 * (__brev(c >> 1) >> (32 - logL1)) + (c & 1)] = acc;
    }
    __syncthreads();
    fft_lines(line, nullptr, twN, L1, logL1);
    for (int i1 = tid; i1 < L1; i1 += bd) {
        const double2 w = i1 == tid ? twk : __ldg(tw + (((int64_t)i2 * i1) & (L - 1)));
        Y[(int64_t)i1 * P.L2 + i2] = cmul(line[i1], w);
    }
    __syncthreads();
}

__device__ __forceinline__ void rows_phase(const DevPlan& P, int64_t n, const double2* Y, double2* T, int k1,
                                           int do_inverse, unsigned char* smraw) {
    const int L1 = P.L1, L2 = P.L2, L = P.L, K = P.K, bd = blockDim.x, tid = threadIdx.x;
    double2* A = (double2*)smraw;
    double2* B = A + L2;
    double2* twN = A + 2 * L2;
    const int logL2 = 31 - __clz(L2);
    const int k1p = (L1 - k1) % L1;
    const bool pair = k1p != k1;
    double2* Bp = pair ? B : A;            // row holding the partners of row k1's modes
    const double2* tw = (const double2*)P.twiddle;
    // first loads together: the two rows and the line twiddles
    for (int i2 = tid; i2 < L2; i2 += bd) {
        int rv = __brev(i2) >> (32 - logL2);
        double2 ya = __ldcg(Y + (int64_t)k1 * L2 + i2);
        double2 yb = pair ? __ldcg(Y + (int64_t)k1p * L2 + i2) : make_double2(0.0, 0.0);
        double2 t = i2 < L2 / 2 ? __ldg(tw + i2 * (L / L2)) : make_double2(0.0, 0.0);
        A[rv] = ya;
        if (pair) B[rv] = yb;
        if (i2 < L2 / 2) twN[i2] = t;
    }
    __syncthreads();
    fft_lines(A, pair ? B : nullptr, twN, L2, logL2);
    // zero the spectrum positions no mode owns (K < index < L - K)
    for (int t = tid; t < 2 * L2; t += bd) {
        int row = t < L2 ? k1 : k1p;
        int k2 = t < L2 ? t : t - L2;
        if (t >= L2 && !pair) break;
        int idx = row + L1 * k2;
        if (idx > K && idx < L - K) (t < L2 ? A : B)[k2] = make_double2(0.0, 0.0);
    }
    // modes of the two rows, one thread per mode; each position of A and B belongs to one mode
    const int nA = k1 <= K ? (K - k1) / L1 + 1 : 0;
    const int nB = (pair && k1p <= K) ? (K - k1p) / L1 + 1 : 0;
    for (int mq = tid; mq < nA + nB; mq += bd) {
        double2* row = A;
        double2* prow = Bp;
        int k2, pos, k;
        if (mq < nA) {
            k2 = mq;
            k = k1 + L1 * k2;
            if (k1 == 0) { prow = A; pos = (L2 - k2) % L2; }
            else pos = L2 - 1 - k2;
        } else {
            row = B;
            prow = A;
            k2 = mq - nA;
            k = k1p + L1 * k2;
            pos = L2 - 1 - k2;
        }
        const double* f = P.modefac + 8 * (int64_t)k;
        const double2 fp = make_double2(__ldg(f + 3), __ldg(f + 4)), fm = make_double2(__ldg(f + 5), __ldg(f + 6));
        const double2 an = mode_update(P, n, k, row[k2], prow[pos]);
        // type-2 spectrum of the mode: Zs[k] = alpha_k deconv2_k (1 + i w^k),
        // Zs[L-k] = conj(alpha_k) deconv2_k (1 - i w^{L-k})
        row[k2] = cmul(an, fp);
        if (k > 0) prow[pos] = cmul(cconj(an), fm);
    }
    __syncthreads();
    if (!do_inverse) return;
    // first pass of the inverse FFT: bit-reverse the rows in place, FFT over k2 with sign -
    for (int i = tid; i < L2; i += bd) {
        int j = __brev(i) >> (32 - logL2);
        if (i < j) {
            double2 t = A[i]; A[i] = A[j]; A[j] = t;
            if (pair) { t = B[i]; B[i] = B[j]; B[j] = t; }
        }
    }
    for (int j = tid; j < L2 / 2; j += bd) twN[j].y = -twN[j].y;
    __syncthreads();
    fft_lines(A, pair ? B : nullptr, twN, L2, logL2);
    for (int i2 = tid; i2 < L2; i2 += bd) {
        double2 w = __ldg(tw + (((int64_t)k1 * i2) & (L - 1)));
        T[(int64_t)k1 * L2 + i2] = cmul(A[i2], cconj(w));
        if (pair) {
            double2 wp = __ldg(tw + (((int64_t)k1p * i2) & (L - 1)));
            T[(int64_t)k1p * L2 + i2] = cmul(B[i2], cconj(wp));
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void icols_phase(const DevPlan& P, const double2* T, int i2, unsigned char* smraw) {
    const int L1 = P.L1, bd = blockDim.x, tid = threadIdx.x;
    double2* sm = (double2*)smraw;
    double2* twN = sm + L1;
    const int logL1 = 31 - __clz(L1);
    const double2* tw = (const double2*)P.twiddle;
    for (int k1 = tid; k1 < L1; k1 += bd) {
        double2 v = __ldcg(T + (int64_t)k1 * P.L2 + i2);
        double2 t = k1 < L1 / 2 ? __ldg(tw + k1 * (P.L / L1)) : make_double2(0.0, 0.0);
        sm[__brev(k1) >> (32 - logL1)] = v;
        if (k1 < L1 / 2) twN[k1] = make_double2(t.x, -t.y);
    }
    __syncthreads();
    fft_lines(sm, nullptr, twN, L1, logL1);
    double2* grid = (double2*)P.grid;
    for (int i1 = tid; i1 < L1; i1 += bd) grid[i2 + (int64_t)P.L2 * i1] = sm[i1];
    __syncthreads();
}

// modes per block of the per-stage FIR tail kernel (one octet of lanes per mode, 256 threads)
constexpr int kTailModes = 32;

// ---------------------------------------------------------------------------------------------
// incident forcing g_j(t) = beta_j f(x_j - t), f periodised over 2 pi in the periodic box (eq. gj).
// pulse[3i..3i+2] = amp, centre, 1/width.  Gaussian terms beyond 12 widths (below e^-72 of the
// amplitude) are skipped.
// ---------------------------------------------------------------------------------------------
__device__ inline double incident(const DevPlan& P, double s) {
    double f = 0.0;
    const double kTwoPi = 6.283185307179586476925286766559;
    const double kInvTwoPi = 0.15915494309189533576888376337251;
    for (int i = 0; i < P.npulse; i++) {
        double amp = P.pulse[3 * i], cen = P.pulse[3 * i + 1], iw = P.pulse[3 * i + 2];
        if (P.bc == WAVE1D_FREE) {
            double z = (s - cen) * iw;
            if (fabs(z) <= 12.0) f += amp * exp(-0.5 * z * z);
        } else {
            double span = 12.0 / iw;
            int64_t m0 = (int64_t)floor((cen - s - span) * kInvTwoPi);
            int64_t m1 = (int64_t)ceil((cen - s + span) * kInvTwoPi);
            for (int64_t m = m0; m <= m1; m++) {
                double z = (s + kTwoPi * (double)m - cen) * iw;
                if (fabs(z) <= 12.0) f += amp * exp(-0.5 * z * z);
            }
        }
    }
    return f;
}

// forcing g_j(t_{n+1}) of spring j: the caller's vector, else beta_j f(x_j - t_{n+1})
__device__ __forceinline__ double forcing(const DevPlan& P, int64_t n, int64_t j) {
    if (P.g_ext) return P.g_ext[j];
    return __ldg(P.beta + j) * incident(P, __ldg(P.x + j) - (double)(n + 1) * P.dt);
}

// ---------------------------------------------------------------------------------------------
// type-2 interpolation: u_H(x_t) = sum_{t'} G'[(i0 + t') mod nf] psi_{t,t'} for springs, then
// receivers; for springs also the forcing and u_H part of the right-hand side of eq. linearSystem,
// rhs_j = -g_j(t_{n+1}) - beta_j u_H(x_j), with g_j from gpre (computed ahead) or computed here.
// One chunk = kInterpPoints points, two threads per point (the first ceil(w/2) taps and the
// rest, each summed in tap order with its loads in one batch, then added), 256 threads.
// ---------------------------------------------------------------------------------------------
constexpr int kInterpPoints = 128;

__device__ __forceinline__ void interp_chunk(const DevPlan& P, int64_t n, int64_t chunk, const double* gpre) {
    const int64_t t = chunk * kInterpPoints + (threadIdx.x >> 1);
    const int half = threadIdx.x & 1;
    const int64_t total = P.M + P.R;
    const int w = P.w, nf = P.nf, wh = (w + 1) >> 1;
    const bool in = t < total;
    const bool spring = t < P.M;
    const int64_t j = spring ? t : t - P.M;
    const int i0 = in ? (spring ? __ldg(P.sp_i0 + j) : __ldg(P.rc_i0 + j)) : 0;
    const double* ker = spring ? P.sp_ker + j * w : P.rc_ker + j * w;
    const double bj = (in && spring) ? __ldg(P.beta + j) : 0.0;
    const double gj = (in && spring && gpre) ? __ldcg(gpre + j) : 0.0;
    const int tb = half ? wh : 0, te = half ? w : wh;
    double acc = 0.0;
    for (int t0 = tb; t0 < te; t0 += 8) {
        double gv[8], kv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            int tt = t0 + u;
            if (in && tt < te) {
                int i = i0 + tt;
                i = i >= nf ? i - nf : i;
                gv[u] = __ldcg(P.grid + i);
                kv[u] = __ldg(ker + tt);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (in && t0 + u < te) acc = fma(gv[u], kv[u], acc);
    }
    const double other = __shfl_xor_sync(0xffffffffu, acc, 1);
    if (!in || half) return;
    acc = acc + other;
    if (spring) {
        P.uH[j] = acc;
        const double g = gpre ? gj : forcing(P, n, j);
        P.rhs[j] = -g - bj * acc;
    } else {
        P.uHr[j] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// Implicit solve of eq. linearSystem, -(I + S) sigma^{n+1} = g + (beta/2) c + beta u_H, with the
// local sum c_j assembled from the partials of row j's items (kept for inspection).
// ---------------------------------------------------------------------------------------------
// rhs_j from the partials of row j's items [a, e), summed in item order (kept in clocal)
__device__ __forceinline__ double rhs_items(const DevPlan& P, int j, int64_t a, int64_t e, double bj) {
    const double rj = __ldcg(P.rhs + j);
    double c = 0.0;
    for (int64_t it = a; it < e; it += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = it + u < e ? __ldcg(P.l_part + it + u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (it + u < e) c += v[u];
    }
    P.clocal[j] = c;
    return fma(-0.5 * bj, c, rj);
}

__device__ __forceinline__ double rhs_of(const DevPlan& P, int j) {
    return rhs_items(P, j, __ldg(P.l_item_ptr + j), __ldg(P.l_item_ptr + j + 1), __ldg(P.beta + j));
}

__device__ __forceinline__ void store_sigma(const DevPlan& P, int64_t n, int j, double v) {
    int slot = ring_slot(n + 1, P.ring);
    P.sig[(int64_t)slot * P.M + j] = v;
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    float2 pr = make_float2(hi, lo);
    ((float2*)P.sig2)[(int64_t)slot * P.M + j] = pr;
    ((float2*)P.sig2)[(int64_t)(slot + P.ring) * P.M + j] = pr;
    if (!isfinite(v)) atomicCAS(P.status, 0, (int)WAVE1D_ENONFINITE);
    if (P.sig_hist) P.sig_hist[(n % P.chunk) * P.M + P.perm[j]] = v;
}

// block solve sigma^{n+1} = (I + S)^{-1} rhs.  The inverse of each block of springs closer than
// dt is stored column-major (invT[l * s + i] = inv[i][l]).  Tasks t = first, first + stride, ...
// (one warp each):
//   t < n_sgroups  a solve group: consecutive blocks of at most 32 members packed into the warp's
//                  lanes (lane = one row); the right-hand sides of a block pass between its lanes
//                  by shuffles, so every FP64 instruction works on up to 32 rows at once
//   otherwise      32 rows of a block of more than 32 members (big_row0 gives the first row);
//                  blocks of up to kSolveStage members stage all their right-hand sides in the
//                  warp's srhs (kSolveStage doubles of shared memory); larger blocks have one
//                  task, which forms the right-hand side in place in P.rhs
// Each row sums over l = 0 .. s-1 in order, even l into one accumulator and odd l into another.
constexpr int kSolveStage = 256;
constexpr int kSolveBatch = 16;

__device__ __forceinline__ void solve_tasks(const DevPlan& P, int64_t n, int64_t first, int64_t stride,
                                            double* srhs) {
    const int lane = threadIdx.x & 31;
    for (int64_t task = first; task < P.n_sgroups + P.n_big; task += stride) {
        if (task < P.n_sgroups) {
            const int64_t e = task * 32 + lane;
            const int j = __ldg(P.sg_j + e);
            const int meta = __ldg(P.sg_meta + e);
            const double* invT = P.inv + __ldg(P.sg_off + e);
            const int smax = __ldg(P.sg_smax + task);
            const double bj = __ldg(P.sg_beta + e);
            const int64_t ip = __ldg(P.sg_ip + e);
            const int icnt = __ldg(P.sg_icnt + e);
            const int b0 = meta & 255, s = (meta >> 8) & 255, i = meta >> 16;
            const double r = j >= 0 ? rhs_items(P, j, ip, ip + icnt, bj) : 0.0;
            double a0 = 0.0, a1 = 0.0;
            for (int l0 = 0; l0 < smax; l0 += kSolveBatch) {
                double v[kSolveBatch];
#pragma unroll
                for (int u = 0; u < kSolveBatch; u++) v[u] = l0 + u < s ? __ldg(invT + (int64_t)(l0 + u) * s + i) : 0.0;
#pragma unroll
                for (int u = 0; u < kSolveBatch; u += 2) {
                    const double r0 = __shfl_sync(0xffffffffu, r, min(b0 + l0 + u, 31));
                    const double r1 = __shfl_sync(0xffffffffu, r, min(b0 + l0 + u + 1, 31));
                    if (l0 + u < s) a0 = fma(v[u], r0, a0);
                    if (l0 + u + 1 < s) a1 = fma(v[u + 1], r1, a1);
                }
            }
            if (j >= 0) store_sigma(P, n, j, a0 + a1);
            continue;
        }
        const int64_t bt = task - P.n_sgroups;
        const int64_t b = __ldg(P.big_blk + bt);
        const int r0 = __ldg(P.big_row0 + bt);
        const int64_t m0 = __ldg(P.blk_ptr + b);
        const int s = (int)(__ldg(P.blk_ptr + b + 1) - m0);
        const double* invT = P.inv + __ldg(P.blk_inv_off + b);
        if (s <= kSolveStage) {
            for (int l0 = 0; l0 < s; l0 += 64) {           // two rows per lane per pass
                const int la = l0 + lane, lb = l0 + 32 + lane;
                const int ja = la < s ? __ldg(P.blk_members + m0 + la) : 0;
                const int jb = lb < s ? __ldg(P.blk_members + m0 + lb) : 0;
                const double ra = la < s ? rhs_of(P, ja) : 0.0;
                const double rb = lb < s ? rhs_of(P, jb) : 0.0;
                if (la < s) srhs[la] = ra;
                if (lb < s) srhs[lb] = rb;
            }
            __syncwarp();
            const int i = r0 + lane;
            if (i < s) {
                double a0 = 0.0, a1 = 0.0;
                for (int l0 = 0; l0 < s; l0 += kSolveBatch) {
                    double v[kSolveBatch];
#pragma unroll
                    for (int u = 0; u < kSolveBatch; u++) v[u] = l0 + u < s ? __ldg(invT + (int64_t)(l0 + u) * s + i) : 0.0;
#pragma unroll
                    for (int u = 0; u < kSolveBatch; u += 2) {
                        if (l0 + u < s) a0 = fma(v[u], srhs[l0 + u], a0);
                        if (l0 + u + 1 < s) a1 = fma(v[u + 1], srhs[l0 + u + 1], a1);
                    }
                }
                store_sigma(P, n, __ldg(P.blk_members + m0 + i), a0 + a1);
            }
            __syncwarp();
        } else {
            // very large blocks (one task): the full right-hand side is formed in place in P.rhs
            for (int i = lane; i < s; i += 32) {
                int j = __ldg(P.blk_members + m0 + i);
                P.rhs[j] = rhs_of(P, j);
            }
            __syncwarp();
            for (int i = lane; i < s; i += 32) {
                double a0 = 0.0, a1 = 0.0;
                for (int l = 0; l < s; l++) {
                    const double x = __ldg(invT + (int64_t)l * s + i);
                    const double rl = __ldcg(P.rhs + __ldg(P.blk_members + m0 + l));
                    if (l & 1) a1 = fma(x, rl, a1);
                    else a0 = fma(x, rl, a0);
                }
                store_sigma(P, n, __ldg(P.blk_members + m0 + i), a0 + a1);
            }
            __syncwarp();
        }
    }
}

// receivers, after every density of the step is stored: u = 1/2 (sum of the receiver row's item
// partials (m >= 1) + sum over sources closer than dt of Q_0 sigma^{n+1}) + u_H; one warp per
// receiver, the m = 0 terms padded to r0_stride lanes (zero weight on padding), run by the block
// that finishes the step last.
__device__ __forceinline__ void receivers_readout(const DevPlan& P, int64_t n) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const double* s1 = P.sig + (int64_t)ring_slot(n + 1, P.ring) * P.M;
    for (int64_t r = wid; r < P.R; r += nwarps) {
        const double uh = __ldcg(P.uHr + r);
        double cr = 0.0;
        for (int64_t it = __ldg(P.r_item_ptr + r) + lane; it < __ldg(P.r_item_ptr + r + 1); it += 32)
            cr += __ldcg(P.r_part + it);
        double acc = 0.0;
        for (int e = lane; e < P.r0_stride; e += 32) {
            const int64_t idx = r * P.r0_stride + e;
            acc = fma(__ldg(P.r0p_w + idx), __ldcg(s1 + __ldg(P.r0p_src + idx)), acc);
        }
        cr = warp_sum(cr);
        acc = warp_sum(acc);
        if (lane == 0) P.rec_hist[(n % P.chunk) * P.R + r] = 0.5 * (cr + acc) + uh;
    }
}

}  // namespace wave1d
