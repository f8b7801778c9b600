// Per-step kernels of the WFP march.  One time step n -> n+1:
//   k_local_items local explicit sum over the last delta of history (Sec. 4.1, m >= 1), on a side
//                 stream, concurrent with the history pipeline
//   history pipeline (history.cu): spreading + forward FFT columns, forward FFT rows + mode
//                 update (Sec. 3) + inverse FFT rows, inverse FFT columns
//   [k_rbc_grid, k_rbc_update, k_fft_cols, k_fft_rows]  on projection steps (Sec. 4.4) the
//                 projection and the inverse FFT of the natural-order type-2 spectrum
//   k_interp      u_H at springs and receivers (eq. historySol1 via NUFFT)
//   k_solve       right-hand side and block solve of eq. linearSystem; its last block reads out
//                 the receivers (u = u_L + u_H) and advances the step counter
// Kernels read the step index n from device memory so that captured graphs can be replayed.
//
// GB300 runs FP64 at about 2 FMA per clock per SM and FP32 at 128, so the one kernel with a
// per-pair inner loop (the local sum) does its products and sums in compensated FP32 pairs
// (hi + lo, about 48 significant bits), which keeps it bound by HBM rather than by the FP64 pipe.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "device_common.cuh"
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
        float4 w01 = __ldg(wp + 32 * (t >> 1)), w23 = __ldg(wp + 32 * ((t >> 1) + 1));
        float4 w45 = __ldg(wp + 32 * ((t >> 1) + 2)), w67 = __ldg(wp + 32 * ((t >> 1) + 3));
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
        float4 w = __ldg(wp + 32 * (t >> 1));
        pair_mac(sh, sl, make_float2(w.x, w.y), __ldg(sp));
        pair_mac(sh, sl, make_float2(w.z, w.w), __ldg(sp - M));
        sp -= 2 * M;
    }
}

// one warp per item, items handed out by an atomic counter (spring items, then receiver items
// with m >= 1); the solve resets the counter after the step's local sums are done
__global__ void __launch_bounds__(256, 4) k_local_items(DevPlan P) {
    int64_t n = load_step(P);
    int lane = threadIdx.x & 31;
    int q = ring_slot(n + 1, P.ring);
    unsigned long long total = (unsigned long long)(P.l_nitems + P.r_nitems);
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(P.item_ctr, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total) break;
        float sh = 0.f, sl = 0.f;
        if (g < (unsigned long long)P.l_nitems) {
            int sj = __ldg(P.l_src + g * 32 + lane);
            local_item((const float2*)P.sig2, P.M, P.ring, q, P.l_mfirst, P.l_s0[g], P.l_len[g],
                       (const float4*)(P.l_w + 2 * P.l_wbase[g]) + lane, sj, sh, sl);
            pair_warp_sum(sh, sl);
            if (lane == 0) P.l_part[g] = (double)sh + (double)sl;
        } else {
            int64_t it = (int64_t)g - P.l_nitems;
            int sj = __ldg(P.r_src + it * 32 + lane);
            local_item((const float2*)P.sig2, P.M, P.ring, q, P.r_mfirst, P.r_s0[it], P.r_len[it],
                       (const float4*)(P.r_w + 2 * P.r_wbase[it]) + lane, sj, sh, sl);
            pair_warp_sum(sh, sl);
            if (lane == 0) P.r_part[it] = (double)sh + (double)sl;
        }
    }
}

// receivers, after every density of the step is stored: u = 1/2 (sum of the m >= 1 item partials
// + sum over sources closer than dt of Q_0 sigma^{n+1}) + u_H; one warp per receiver, run by the
// last block of k_solve to finish.
__device__ __forceinline__ void receivers_readout(const DevPlan& P, int64_t n) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const double* s1 = P.sig + (int64_t)ring_slot(n + 1, P.ring) * P.M;
    for (int64_t r = wid; r < P.R; r += nwarps) {
        double acc = 0.0;
        for (int64_t it = P.r_item_ptr[r] + lane; it < P.r_item_ptr[r + 1]; it += 32) acc += P.r_part[it];
        for (int64_t e = P.r0_ptr[r] + lane; e < P.r0_ptr[r + 1]; e += 32)
            acc = fma(P.r0_w[e], __ldcg(s1 + P.r0_src[e]), acc);
        acc = warp_sum(acc);
        if (lane == 0) P.rec_hist[(n % P.chunk) * P.R + r] = 0.5 * acc + P.uHr[r];
    }
}

// ---------------------------------------------------------------------------------------------
// Complex FFT of length L = L1 * L2 (powers of two), X[k] = sum_i z[i] e^{sign 2 pi i ik/L}:
//   columns: for each i2, FFT over i1 of z[i2 + L2 i1], times e^{sign 2 pi i i2 k1/L} -> Y[k1 L2 + i2]
//   rows:    for each k1, FFT over i2 of Y[k1 L2 + i2] -> X[k1 + L1 k2]
// Each block transforms one line in shared memory: bit-reversed load, radix-2 DIT stages with the
// line's N/2 twiddles staged in shared memory.  tw[j] = e^{+2 pi i j / L}.
// ---------------------------------------------------------------------------------------------
__global__ void k_fft_cols(const double2* __restrict__ in, double2* __restrict__ out,
                           const double2* __restrict__ tw, int L, int L1, int L2, int logL1, int sign) {
    extern __shared__ double2 sm[];
    double2* twN = sm + L1;
    int i2 = blockIdx.x;
    stage_twiddles(twN, tw, L, L1, sign);
    for (int i1 = threadIdx.x; i1 < L1; i1 += blockDim.x)
        sm[__brev(i1) >> (32 - logL1)] = in[i2 + (int64_t)L2 * i1];
    __syncthreads();
    fft_line(sm, twN, L1, logL1);
    for (int k1 = threadIdx.x; k1 < L1; k1 += blockDim.x) {
        int idx = (int)(((int64_t)i2 * k1) % L);
        double2 w = tw[idx];
        if (sign < 0) w.y = -w.y;
        out[(int64_t)k1 * L2 + i2] = cmul(sm[k1], w);
    }
}

__global__ void k_fft_rows(const double2* __restrict__ in, double2* __restrict__ out,
                           const double2* __restrict__ tw, int L, int L1, int L2, int logL2, int sign) {
    extern __shared__ double2 sm[];
    double2* twN = sm + L2;
    int k1 = blockIdx.x;
    stage_twiddles(twN, tw, L, L2, sign);
    for (int i2 = threadIdx.x; i2 < L2; i2 += blockDim.x)
        sm[__brev(i2) >> (32 - logL2)] = in[(int64_t)k1 * L2 + i2];
    __syncthreads();
    fft_line(sm, twN, L2, logL2);
    for (int k2 = threadIdx.x; k2 < L2; k2 += blockDim.x) out[k1 + (int64_t)L1 * k2] = sm[k2];
}

// ---------------------------------------------------------------------------------------------
// Radiation projection (Sec. 4.4), applied to alpha^{n+1}, alpha'^{n+1} on projection steps.
// The 2K-point grid values of the real field with modes |k| <= K-1 change only at the 4W points
// next to x = +-pi, so the projected coefficients are
//   alpha_k + (1/2K) sum_{i in I} du_i e^{+i k x_i},  alpha'_k + (1/2K) sum_{i in I} dv_i e^{+i k x_i}
// with du = (phi_s - 1) u, dv = phi_s' u + (phi_s - 1) v (eq. vtilde), and alpha_K = 0.
// x_i = i pi/K, so e^{i k x_i} = tw2K[k i mod 2K] (exact argument reduction).
// ---------------------------------------------------------------------------------------------
__global__ void k_rbc_grid(DevPlan P) {
    int pt = blockIdx.x;                     // one block per rolled-off grid point
    int ig = P.rbc_idx[pt];
    const double2* al = (const double2*)P.alpha;
    const double2* alp = (const double2*)P.alpha_p;
    const double2* t2 = (const double2*)P.tw2K;
    int64_t twoK = 2 * (int64_t)P.K;
    double su = 0.0, sv = 0.0;
    int k = 1 + threadIdx.x;
    int64_t a = ((int64_t)k * ig) % twoK;
    int64_t inc = ((int64_t)blockDim.x * ig) % twoK;
    for (; k < P.K; k += blockDim.x) {
        double2 e = cconj(t2[a]);                     // e^{-i k x}
        su += cmul(al[k], e).x;
        sv += cmul(alp[k], e).x;
        a += inc;
        if (a >= twoK) a -= twoK;
    }
    __shared__ double red[2][32];
    su = warp_sum(su);
    sv = warp_sum(sv);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = su; red[1][wid] = sv; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0, v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { u += red[0][w]; v += red[1][w]; }
        u = al[0].x + 2.0 * u;
        v = alp[0].x + 2.0 * v;
        double ph = P.rbc_phi[pt], dph = P.rbc_dphi[pt];
        P.rbc_uv[4 * pt + 0] = u;
        P.rbc_uv[4 * pt + 1] = v;
        P.rbc_uv[4 * pt + 2] = (ph - 1.0) * u;
        P.rbc_uv[4 * pt + 3] = fma(dph, u, (ph - 1.0) * v);
    }
}

__global__ void k_rbc_update(DevPlan P, int npts) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > P.K) return;
    double2* al = (double2*)P.alpha;
    double2* alp = (double2*)P.alpha_p;
    const double2* t2 = (const double2*)P.tw2K;
    double2 a, ap;
    if (k == P.K) {
        a = make_double2(0.0, 0.0);
        ap = a;
    } else {
        double2 du = make_double2(0.0, 0.0), dv = make_double2(0.0, 0.0);
        int64_t twoK = 2 * (int64_t)P.K;
        for (int pt = 0; pt < npts; pt++) {
            double2 e = t2[((int64_t)k * P.rbc_idx[pt]) % twoK];
            double xu = P.rbc_uv[4 * pt + 2], xv = P.rbc_uv[4 * pt + 3];
            du.x = fma(xu, e.x, du.x);
            du.y = fma(xu, e.y, du.y);
            dv.x = fma(xv, e.x, dv.x);
            dv.y = fma(xv, e.y, dv.y);
        }
        double inv = 1.0 / (double)twoK;
        a = al[k];
        ap = alp[k];
        a = make_double2(fma(du.x, inv, a.x), fma(du.y, inv, a.y));
        ap = make_double2(fma(dv.x, inv, ap.x), fma(dv.y, inv, ap.y));
    }
    al[k] = a;
    alp[k] = ap;
    write_type2(P, k, a, (double2*)P.spec2);
}

__device__ double incident(const DevPlan& P, double s);

// ---------------------------------------------------------------------------------------------
// type-2 interpolation: u_H(x_t) = sum_{t'} G'[(i0 + t') mod nf] psi_{t,t'} for springs, then
// receivers; for springs also the forcing and u_H part of the right-hand side of eq. linearSystem.
// ---------------------------------------------------------------------------------------------
__global__ void k_interp(DevPlan P) {
    int64_t total = P.M + P.R;
    const int w = P.w, nf = P.nf;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        bool spring = t < P.M;
        int64_t j = spring ? t : t - P.M;
        int i0 = spring ? P.sp_i0[j] : P.rc_i0[j];
        const double* ker = spring ? P.sp_ker + j * w : P.rc_ker + j * w;
        double bj = 0.0, xj = 0.0, gj = 0.0;
        if (spring) {
            bj = P.beta[j];
            if (P.g_ext) gj = P.g_ext[j];
            else xj = P.x[j];
        }
        // taps in batches of 16, loaded before they are summed (in tap order)
        double acc = 0.0;
        for (int t0 = 0; t0 < w; t0 += 16) {
            double gv[16], kv[16];
#pragma unroll
            for (int u = 0; u < 16; u++) {
                int tt = t0 + u;
                if (tt < w) {
                    int i = i0 + tt;
                    i = i >= nf ? i - nf : i;
                    gv[u] = P.grid[i];
                    kv[u] = ker[tt];
                }
            }
#pragma unroll
            for (int u = 0; u < 16; u++)
                if (t0 + u < w) acc = fma(gv[u], kv[u], acc);
        }
        if (spring) {
            P.uH[j] = acc;
            double g = P.g_ext ? gj : bj * incident(P, xj - (double)(load_step(P) + 1) * P.dt);
            P.rhs[j] = -g - bj * acc;
        } else {
            P.uHr[j] = acc;
        }
    }
}

// incident forcing g_j(t) = beta_j f(x_j - t), f periodised over 2 pi in the periodic box (eq. gj).
// pulse[3i..3i+2] = amp, centre, 1/width.  Gaussian terms beyond 12 widths (below e^-72 of the
// amplitude) are skipped.
__device__ double incident(const DevPlan& P, double s) {
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

// right-hand side of eq. linearSystem, rhs_j = -g_j - (beta_j/2) c_j - beta_j u_H(x_j): the part
// without the local sum is formed by k_interp (one thread per spring); the solve adds the local sum
// c_j, assembled from the partials of the row's items (and kept for inspection)
__device__ __forceinline__ double rhs_of(const DevPlan& P, int j) {
    int64_t a = P.l_item_ptr[j], e = P.l_item_ptr[j + 1];
    double bj = P.beta[j], rj = P.rhs[j];
    double c = 0.0;
    for (int64_t it = a; it < e; it += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = it + u < e ? P.l_part[it + u] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (it + u < e) c += v[u];
    }
    P.clocal[j] = c;
    return fma(-0.5 * bj, c, rj);
}

__device__ __forceinline__ void store_sigma(const DevPlan& P, int64_t n, int j, double v) {
    int slot = ring_slot(n + 1, P.ring);
    P.sig[(int64_t)slot * P.M + j] = v;
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    float2 pr = make_float2(hi, lo);
    ((float2*)P.sig2)[(int64_t)slot * P.M + j] = pr;
    ((float2*)P.sig2)[(int64_t)(slot + P.ring) * P.M + j] = pr;
    if (!isfinite(v)) atomicExch(P.status, (int)WAVE1D_ENONFINITE);
    if (P.sig_hist) P.sig_hist[(n % P.chunk) * P.M + P.perm[j]] = v;
}

// block solve sigma^{n+1} = (I + S)^{-1} rhs, one warp per block of springs closer than dt.
// The inverse is stored column-major (invT[l * s + i] = inv[i][l]) so lanes read it contiguously;
// blocks of up to kSolveStage members stage their right-hand sides in the warp's shared memory.
constexpr int kSolveStage = 256;

__global__ void __launch_bounds__(256) k_solve(DevPlan P) {
    __shared__ double srhs[8][kSolveStage];
    __shared__ bool last;
    int64_t n = load_step(P);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.item_ctr = 0ull;   // the step's local sums are done
    if (b < P.nblocks) {
        int64_t m0 = P.blk_ptr[b];
        int s = (int)(P.blk_ptr[b + 1] - m0);
        const double* invT = P.inv + P.blk_inv_off[b];
        if (s <= kSolveStage) {
            double* r = srhs[wid];
            // the first eight inverse entries of the lane's first row load with the members
            double pre[8];
#pragma unroll
            for (int u = 0; u < 8; u++) pre[u] = (lane < s && u < s) ? invT[(int64_t)u * s + lane] : 0.0;
            for (int i = lane; i < s; i += 32) r[i] = rhs_of(P, P.blk_members[m0 + i]);
            __syncwarp();
            for (int i = lane; i < s; i += 32) {
                double a0 = 0.0, a1 = 0.0;
                for (int l0 = 0; l0 < s; l0 += 8) {
                    double v[8];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        v[u] = (l0 == 0 && i == lane) ? pre[u]
                                                      : (l0 + u < s ? invT[(int64_t)(l0 + u) * s + i] : 0.0);
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        if (l0 + u < s) a0 = fma(v[u], r[l0 + u], a0);
                        if (l0 + u + 1 < s) a1 = fma(v[u + 1], r[l0 + u + 1], a1);
                    }
                }
                store_sigma(P, n, P.blk_members[m0 + i], a0 + a1);
            }
        } else {
            // large blocks: the full right-hand side is formed in place in P.rhs first
            for (int i = lane; i < s; i += 32) {
                int j = P.blk_members[m0 + i];
                P.rhs[j] = rhs_of(P, j);
            }
            __syncwarp();
            for (int i = lane; i < s; i += 32) {
                double acc = 0.0;
                for (int l = 0; l < s; l++)
                    acc = fma(invT[(int64_t)l * s + i], P.rhs[P.blk_members[m0 + l]], acc);
                store_sigma(P, n, P.blk_members[m0 + i], acc);
            }
        }
    }
    // the block that finishes last reads out the receivers and advances the step counter (every
    // other block has stored its densities and read n before it counts itself done)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long done = atomicAdd((unsigned long long*)&P.step[1], 1ull);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    receivers_readout(P, n);
    __syncthreads();
    if (threadIdx.x == 0) {
        P.step[1] = 0;
        __threadfence();
        P.step[0] = n + 1;
    }
}

// caller-order gathers and scatters
__global__ void k_sigma_to_caller(DevPlan P, int64_t q, double* out) {
    const double* sg = P.sig + (int64_t)ring_slot(q, P.ring) * P.M;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x)
        out[P.perm[j]] = sg[j];
}

__global__ void k_internal_to_caller(const int32_t* perm, int64_t M, const double* in, double* out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
        out[perm[j]] = in[j];
}

__global__ void k_caller_to_internal(const int32_t* perm, int64_t M, const double* in, double* out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = in[perm[j]];
}

}  // namespace wave1d
