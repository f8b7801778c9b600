// Device helpers shared by the step kernels (complex arithmetic, ring slots, shared-memory FFT
// lines, the type-2 spectrum of one mode, the per-mode update of Sec. 3).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace wave1d {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ int ring_slot(int64_t q, int ring) {
    int64_t r = q % ring;
    return (int)(r < 0 ? r + ring : r);
}

__device__ __forceinline__ int64_t load_step(const DevPlan& P) {
    return *((const volatile int64_t*)P.step);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// radix-2 DIT FFT of one line of N points held in shared memory in bit-reversed order; twN holds
// the line's N/2 twiddles e^{sign 2 pi i j / N}.  All threads of the block take part.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void fft_line(double2* a, const double2* twN, int N, int logN) {
    for (int s = 1; s <= logN; s++) {
        int half = 1 << (s - 1);
        int step = N / (2 * half);
        for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
            int pos = j & (half - 1);
            int i0 = ((j >> (s - 1)) << s) + pos;
            int i1 = i0 + half;
            double2 t = cmul(twN[pos * step], a[i1]);
            double2 u = a[i0];
            a[i0] = cadd(u, t);
            a[i1] = csub(u, t);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void stage_twiddles(double2* twN, const double2* tw, int L, int N, int sign) {
    int stride = L / N;
    for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
        double2 w = tw[j * stride];
        if (sign < 0) w.y = -w.y;
        twN[j] = w;
    }
}

// ---------------------------------------------------------------------------------------------
// Type-2 spectrum of mode k for the inverse real FFT (factors precomputed in modefac):
//   Zs[k] = alpha_k deconv2_k (1 + i w^k),  Zs[L-k] = conj(alpha_k) deconv2_k (1 - i w^{L-k}),
//   w = e^{-2 pi i / nf}; entries with K < idx < L - K stay zero.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void write_type2(const DevPlan& P, int k, double2 a, double2* Zs) {
    const double* f = P.modefac + 8 * (int64_t)k;
    Zs[k] = cmul(a, make_double2(f[3], f[4]));
    if (k > 0) Zs[P.L - k] = cmul(cconj(a), make_double2(f[5], f[6]));
}

// ---------------------------------------------------------------------------------------------
// One mode of the history update, computed by a quad of four lanes (all four call it with the same
// k, Z_k and Z_{L-k}; valid = false for padding quads, which still take part in the shuffles):
//   S_k^n = deconv1_k E_k + deconv1_k e^{2 pi i k/nf} O_k  (E, O from the half-length FFT),
//   h_k = sum_m dt p_k(m dt) S_k^{n-m}, g_k likewise (eq. hkcompdisc), the m sum split over the quad,
//   alpha, alpha' rotated and driven (eq. alphakEvolutionFormulas).
// Lane q == 0 of a valid quad stores S_k^n, alpha_k, alpha'_k and returns alpha_k^{n+1}.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double2 mode_step(const DevPlan& P, int64_t n, int k, bool valid, int q,
                                             double2 zk, double2 zm) {
    int kk = valid ? k : P.K;
    const double* f = P.modefac + 8 * (int64_t)kk;
    double2* al = (double2*)P.alpha;
    double2* alp = (double2*)P.alpha_p;
    // everything the mode needs besides the FIR taps, loaded before them
    double f0 = f[0], f1 = f[1], f2 = f[2];
    double2 a = al[kk], ap = alp[kk];
    double cs = P.rot[3 * kk], so = P.rot[3 * kk + 1], ks = P.rot[3 * kk + 2];
    double2 E = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    double2 D = make_double2(0.5 * (zk.x - zm.x), 0.5 * (zk.y + zm.y));
    double2 O = make_double2(D.y, -D.x);
    double2 Sn = cadd(make_double2(f0 * E.x, f0 * E.y), cmul(make_double2(f1, f2), O));
    const int K1 = P.K + 1, W = P.W;
    double2* Sring = (double2*)P.Sring;
    const double2* pq = (const double2*)P.pq;
    double2 h = make_double2(0.0, 0.0), g = make_double2(0.0, 0.0);
    // taps m = q, q + 4, ...: a batch of eight is loaded before any is used
    int slot = ring_slot(n - q, W);
    for (int m0 = q; m0 < W; m0 += 32) {
        double2 Sv[8], wv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            int m = m0 + 4 * u;
            int sl = slot - 4 * u;
            sl = sl < 0 ? sl + W : sl;
            sl = sl < 0 ? sl + W : sl;
            if (m < W) {
                Sv[u] = (m == 0) ? Sn : Sring[(int64_t)sl * K1 + kk];
                wv[u] = pq[(int64_t)m * K1 + kk];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            if (m0 + 4 * u < W) {
                h.x = fma(wv[u].x, Sv[u].x, h.x);
                h.y = fma(wv[u].x, Sv[u].y, h.y);
                g.x = fma(wv[u].y, Sv[u].x, g.x);
                g.y = fma(wv[u].y, Sv[u].y, g.y);
            }
        }
        slot -= 32 % W;
        slot = slot < 0 ? slot + W : slot;
    }
    for (int o = 1; o < 4; o <<= 1) {
        h.x += __shfl_xor_sync(0xffffffffu, h.x, o);
        h.y += __shfl_xor_sync(0xffffffffu, h.y, o);
        g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
    }
    double2 an = make_double2(0.0, 0.0);
    if (valid && q == 0) {
        Sring[(int64_t)ring_slot(n, W) * K1 + k] = Sn;
        an = make_double2(fma(a.x, cs, fma(ap.x, so, h.x)), fma(a.y, cs, fma(ap.y, so, h.y)));
        double2 apn = make_double2(fma(ap.x, cs, fma(-a.x, ks, g.x)), fma(ap.y, cs, fma(-a.y, ks, g.y)));
        al[k] = an;
        alp[k] = apn;
    }
    return an;
}

}  // namespace wave1d
