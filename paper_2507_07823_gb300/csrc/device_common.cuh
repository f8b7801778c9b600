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

// The same transform of one or two lines (b may be null) with two threads per butterfly: the
// thread of component c (0 = real, 1 = imaginary) reads and writes only component c, taking the
// other component of the product from its neighbour lane.  GB300 issues one FP64 warp
// instruction per 64 cycles per SM partition, so halving the FP64 instructions of each thread and
// doubling the warps that share them shortens every stage.  N >= 16, blockDim a multiple of 32.
__device__ __forceinline__ void fft_lines(double2* a, double2* b, const double2* twN, int N, int logN) {
    const int total = (b ? 2 : 1) * N;          // one thread per (line, butterfly, component)
    if (total & 31) {                           // lines too short to fill whole warps
        fft_line(a, twN, N, logN);
        if (b) fft_line(b, twN, N, logN);
        return;
    }
    for (int s = 1; s <= logN; s++) {
        const int half = 1 << (s - 1);
        const int step = N >> s;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const bool second = t >= N;
            double* x = (double*)(second ? b : a);
            const int tt = second ? t - N : t;
            const int j = tt >> 1, c = tt & 1;
            const int pos = j & (half - 1);
            const int i0 = ((j >> (s - 1)) << s) + pos;
            const int i1 = i0 + half;
            const double2 w = twN[pos * step];
            const double ac = x[2 * i1 + c];                          // own component of a[i1]
            const double ao = __shfl_xor_sync(0xffffffffu, ac, 1);   // the other one
            const double u = x[2 * i0 + c];
            // c = 0: Re(w a) = w.x a.x - w.y a.y;  c = 1: Im(w a) = w.x a.y + w.y a.x.  The sign of
            // w.y is flipped with an integer XOR, which keeps it off the FP64 pipe.
            const double wy = __longlong_as_double(__double_as_longlong(w.y) ^
                                                   (c ? 0ll : (long long)0x8000000000000000ull));
            const double tc = fma(w.x, ac, wy * ao);
            x[2 * i0 + c] = u + tc;
            x[2 * i1 + c] = u - tc;
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
// One mode of the history update (eqs. hkcompdisc, alphakEvolutionFormulas), one thread per mode:
//   S_k^n = deconv1_k E_k + deconv1_k e^{2 pi i k/nf} O_k  (E, O from the half-length FFT),
//   h_k = dt p_k(0) S_k^n + tail_h,  g_k = dt q_k(0) S_k^n + tail_g,
// where the tail (taps m = 1 .. W-1, which need only S^{< n}) was summed by fir_tail earlier in
// the step; then alpha, alpha' are rotated and driven.  Stores S_k^n, alpha_k, alpha'_k and
// returns alpha_k^{n+1}.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double2 mode_update(const DevPlan& P, int64_t n, int k, double2 zk, double2 zm) {
    const double* f = P.modefac + 8 * (int64_t)k;
    double2* al = (double2*)P.alpha;
    double2* alp = (double2*)P.alpha_p;
    const int K1 = P.K + 1;
    const double f0 = f[0], f1 = f[1], f2 = f[2];
    const double2 a = al[k], ap = alp[k];
    const double cs = P.rot[3 * k], so = P.rot[3 * k + 1], ks = P.rot[3 * k + 2];
    const double2 w0 = ((const double2*)P.pq)[k];                 // dt (p_k(0), q_k(0))
    const double2 th = __ldcg((const double2*)P.ftail + 2 * k);   // tail_h
    const double2 tg = __ldcg((const double2*)P.ftail + 2 * k + 1); // tail_g
    const double2 E = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    const double2 D = make_double2(0.5 * (zk.x - zm.x), 0.5 * (zk.y + zm.y));
    const double2 O = make_double2(D.y, -D.x);
    const double2 Sn = cadd(make_double2(f0 * E.x, f0 * E.y), cmul(make_double2(f1, f2), O));
    const double2 h = make_double2(fma(w0.x, Sn.x, th.x), fma(w0.x, Sn.y, th.y));
    const double2 g = make_double2(fma(w0.y, Sn.x, tg.x), fma(w0.y, Sn.y, tg.y));
    ((double2*)P.Sring)[(int64_t)ring_slot(n, P.W) * K1 + k] = Sn;
    const double2 an = make_double2(fma(a.x, cs, fma(ap.x, so, h.x)), fma(a.y, cs, fma(ap.y, so, h.y)));
    const double2 apn = make_double2(fma(ap.x, cs, fma(-a.x, ks, g.x)), fma(ap.y, cs, fma(-a.y, ks, g.y)));
    al[k] = an;
    alp[k] = apn;
    return an;
}

// ---------------------------------------------------------------------------------------------
// FIR tail of step n (eq. hkcompdisc without its m = 0 term), from earlier steps only:
//   tail_h = sum_{m=1}^{W-1} dt p_k(m dt) S_k^{n-m},  tail_g likewise with q_k,
// one octet of lanes per mode: lane q of the octet takes m = 1 + q, 9 + q, ... (five taps for
// W <= 41, loaded at once), and the eight partial sums are added in a fixed tree.  S^{n-m} sits
// in ring slot (n-m) mod W.  All 32 lanes of the warp call it (valid = false for padding lanes).
// ---------------------------------------------------------------------------------------------
constexpr int kTapBatch = 5;

__device__ __forceinline__ void fir_tail(const DevPlan& P, int64_t n, int k, bool valid) {
    const int q = threadIdx.x & 7;
    const int kk = valid ? k : P.K;
    const int K1 = P.K + 1, W = P.W;
    const double2* Sring = (const double2*)P.Sring;
    const double2* pq = (const double2*)P.pq;
    double2 h = make_double2(0.0, 0.0), g = make_double2(0.0, 0.0);
    int slot = ring_slot(n - 1 - q, W);        // slot of m = 1 + q: (n - m) mod W
    for (int m0 = 1 + q; m0 < W; m0 += 8 * kTapBatch) {
        double2 Sv[kTapBatch], wv[kTapBatch];
#pragma unroll
        for (int u = 0; u < kTapBatch; u++) {
            int m = m0 + 8 * u;
            int sl = slot - 8 * u;
            sl = sl < 0 ? sl + W : sl;
            if (m < W) {
                Sv[u] = __ldg(Sring + (int64_t)sl * K1 + kk);
                wv[u] = __ldg(pq + (int64_t)m * K1 + kk);
            }
        }
#pragma unroll
        for (int u = 0; u < kTapBatch; u++) {
            if (m0 + 8 * u < W) {
                h.x = fma(wv[u].x, Sv[u].x, h.x);
                h.y = fma(wv[u].x, Sv[u].y, h.y);
                g.x = fma(wv[u].y, Sv[u].x, g.x);
                g.y = fma(wv[u].y, Sv[u].y, g.y);
            }
        }
        slot -= (8 * kTapBatch) % W;
        slot = slot < 0 ? slot + W : slot;
    }
    for (int o = 1; o < 8; o <<= 1) {
        h.x += __shfl_xor_sync(0xffffffffu, h.x, o);
        h.y += __shfl_xor_sync(0xffffffffu, h.y, o);
        g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
    }
    if (valid && q == 0) {
        ((double2*)P.ftail)[2 * k] = h;
        ((double2*)P.ftail)[2 * k + 1] = g;
    }
}

}  // namespace wave1d
