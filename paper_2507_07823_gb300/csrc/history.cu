// Fused history pipeline of one ordinary step (no radiation projection): the type-1 NUFFT, the
// mode update of Sec. 3 and the type-2 NUFFT's FFT in three kernels instead of seven.
//
// The fine grid of nf reals is viewed as L = nf/2 complex points z[r] = G[2r] + i G[2r+1], and
// L = L1 L2 with r = i2 + L2 i1 (column i2) and k = k1 + L1 k2 (row k1).
//   k_hist_cols  spreading of sigma^n into the column's points (eq. densco), FFT over i1 (sign +),
//                twiddle e^{+2 pi i i2 k1/L}  ->  Y[k1 L2 + i2]
//   k_hist_rows  rows k1 and L1 - k1 together: FFT over i2 -> Z_k for k = k1 + L1 k2; the modes of
//                the two rows (each needs Z_k and Z_{L-k}, which lie in the pair) are advanced
//                (eqs. hkcompdisc, alphakEvolutionFormulas) and replaced by their type-2 spectrum;
//                then the first pass of the inverse FFT: FFT over k2 (sign -), twiddle
//                e^{-2 pi i k1 i2/L}  ->  T[k1 L2 + i2]
//   k_hist_icols FFT over k1 (sign -) of T[k1 L2 + i2]  ->  z'[i2 + L2 i1], i.e. the grid G'.
// On projection steps k_hist_rows stops after the mode update and the unfused inverse path runs.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"
#include "internal.h"

namespace wave1d {

// The column's spreading entries are one contiguous range (rows in column-pass order): all threads
// stage the products g_w[e] sigma_{g_src[e]} of a chunk of that range in shared memory with
// independent loads, then thread i1 sums the sub-ranges of its two reals in entry order.
__device__ __forceinline__ void sum_range(const double* prod, int base, int cend, int e0, int e1,
                                          double& a0, double& a1) {
    int lo = max(e0, base), hi = min(e1, cend);
    for (int e = lo; e < hi; e++) {
        if ((e - e0) & 1) a1 += prod[e - base];
        else a0 += prod[e - base];
    }
}

__global__ void k_hist_cols(DevPlan P, double2* __restrict__ Y) {
    extern __shared__ double2 sm[];
    const int L1 = P.L1;
    double2* twN = sm + L1;
    double* prod = (double*)(twN + L1 / 2);
    int64_t n = load_step(P);
    const double* sg = P.sig + (int64_t)ring_slot(n, P.ring) * P.M;
    int i2 = blockIdx.x;
    int logL1 = 31 - __clz(L1);
    const int32_t* ptr = P.g_ptr + (int64_t)i2 * 2 * L1;
    const double2* tw = (const double2*)P.twiddle;
    int i1 = threadIdx.x;
    bool own = i1 < L1;
    int e0 = 0, e1 = 0, e2 = 0;
    double2 twk = make_double2(1.0, 0.0);
    if (own) {
        e0 = ptr[2 * i1];
        e1 = ptr[2 * i1 + 1];
        e2 = ptr[2 * i1 + 2];
        twk = tw[((int64_t)i2 * i1) % P.L];
    }
    int c0 = ptr[0], c1 = ptr[2 * L1];
    if (threadIdx.x < L1 / 2) twN[threadIdx.x] = tw[threadIdx.x * (P.L / L1)];
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    for (int base = c0; base < c1; base += kSpreadChunk) {
        int cend = min(c1, base + kSpreadChunk);
        int e = base + threadIdx.x;
        const int stride = blockDim.x;
        for (; e + 3 * stride < cend; e += 4 * stride) {
            int s0 = __ldg(P.g_src + e), s1 = __ldg(P.g_src + e + stride);
            int s2 = __ldg(P.g_src + e + 2 * stride), s3 = __ldg(P.g_src + e + 3 * stride);
            double w0 = __ldg(P.g_w + e), w1 = __ldg(P.g_w + e + stride);
            double w2 = __ldg(P.g_w + e + 2 * stride), w3 = __ldg(P.g_w + e + 3 * stride);
            double v0 = sg[s0], v1 = sg[s1], v2 = sg[s2], v3 = sg[s3];
            prod[e - base] = w0 * v0;
            prod[e + stride - base] = w1 * v1;
            prod[e + 2 * stride - base] = w2 * v2;
            prod[e + 3 * stride - base] = w3 * v3;
        }
        for (; e < cend; e += stride) prod[e - base] = __ldg(P.g_w + e) * sg[__ldg(P.g_src + e)];
        __syncthreads();
        if (own) {
            sum_range(prod, base, cend, e0, e1, a0, a1);
            sum_range(prod, base, cend, e1, e2, b0, b1);
        }
        __syncthreads();
    }
    if (own) sm[__brev(i1) >> (32 - logL1)] = make_double2(a0 + a1, b0 + b1);
    __syncthreads();
    fft_line(sm, twN, L1, logL1);
    if (own) Y[(int64_t)i1 * P.L2 + i2] = cmul(sm[i1], twk);
}

// position of mode index k in its row: k1 = k mod L1, k2 = k / L1
__global__ void k_hist_rows(DevPlan P, const double2* __restrict__ Y, double2* __restrict__ T,
                            int do_inverse) {
    extern __shared__ double2 sm[];
    const int L1 = P.L1, L2 = P.L2, L = P.L, K = P.K;
    double2* A = sm;
    double2* B = sm + L2;
    double2* twN = sm + 2 * L2;
    int64_t n = load_step(P);
    int logL2 = 31 - __clz(L2);
    int k1 = blockIdx.x;                   // 0 .. L1/2
    int k1p = (L1 - k1) % L1;
    bool pair = k1p != k1;
    double2* Bp = pair ? B : A;            // row holding the partners of row k1's modes
    const double2* tw = (const double2*)P.twiddle;
    // first loads together: the two rows, the line twiddles and the inverse pass's twiddles of
    // this thread's first column
    double2 wi = make_double2(1.0, 0.0), wip = make_double2(1.0, 0.0);
    if (do_inverse && threadIdx.x < L2) {
        wi = tw[((int64_t)k1 * threadIdx.x) % L];
        wip = tw[((int64_t)k1p * threadIdx.x) % L];
    }
    for (int i2 = threadIdx.x; i2 < L2; i2 += blockDim.x) {
        int rv = __brev(i2) >> (32 - logL2);
        double2 ya = Y[(int64_t)k1 * L2 + i2];
        double2 yb = pair ? Y[(int64_t)k1p * L2 + i2] : make_double2(0.0, 0.0);
        double2 t = i2 < L2 / 2 ? tw[i2 * (L / L2)] : make_double2(0.0, 0.0);
        A[rv] = ya;
        if (pair) B[rv] = yb;
        if (i2 < L2 / 2) twN[i2] = t;
    }
    __syncthreads();
    fft_line(A, twN, L2, logL2);
    if (pair) fft_line(B, twN, L2, logL2);
    // zero the spectrum positions no mode owns (K < index < L - K)
    for (int t = threadIdx.x; t < 2 * L2; t += blockDim.x) {
        int row = t < L2 ? k1 : k1p;
        int k2 = t < L2 ? t : t - L2;
        if (t >= L2 && !pair) break;
        int idx = row + L1 * k2;
        if (idx > K && idx < L - K) (t < L2 ? A : B)[k2] = make_double2(0.0, 0.0);
    }
    // modes of the two rows, one quad of lanes per mode
    int nA = k1 <= K ? (K - k1) / L1 + 1 : 0;
    int nB = (pair && k1p <= K) ? (K - k1p) / L1 + 1 : 0;
    int nmodes = nA + nB;
    int quads = blockDim.x >> 2;
    int q = threadIdx.x & 3;
    for (int base = 0; base < nmodes; base += quads) {
        int mq = base + (threadIdx.x >> 2);
        bool valid = mq < nmodes;
        double2* row = A;
        double2* prow = Bp;
        int k2 = 0, pos = 0, k = K;
        if (valid) {
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
        }
        double2 zk = valid ? row[k2] : make_double2(0.0, 0.0);
        double2 zm = valid ? prow[pos] : make_double2(0.0, 0.0);
        const double* f = P.modefac + 8 * (int64_t)(valid ? k : K);
        double2 fp = make_double2(f[3], f[4]), fm = make_double2(f[5], f[6]);
        double2 an = mode_step(P, n, k, valid, q, zk, zm);
        if (valid && q == 0) {
            row[k2] = cmul(an, fp);
            if (k > 0) prow[pos] = cmul(cconj(an), fm);
        }
    }
    if (!do_inverse) return;
    __syncthreads();
    // first pass of the inverse FFT: bit-reverse the rows in place, FFT over k2 with sign -
    for (int i = threadIdx.x; i < L2; i += blockDim.x) {
        int j = __brev(i) >> (32 - logL2);
        if (i < j) {
            double2 t = A[i]; A[i] = A[j]; A[j] = t;
            if (pair) { t = B[i]; B[i] = B[j]; B[j] = t; }
        }
    }
    for (int j = threadIdx.x; j < L2 / 2; j += blockDim.x) twN[j].y = -twN[j].y;
    __syncthreads();
    fft_line(A, twN, L2, logL2);
    if (pair) fft_line(B, twN, L2, logL2);
    for (int i2 = threadIdx.x; i2 < L2; i2 += blockDim.x) {
        bool first = i2 == (int)threadIdx.x;
        double2 w = first ? wi : tw[((int64_t)k1 * i2) % L];
        T[(int64_t)k1 * L2 + i2] = cmul(A[i2], cconj(w));
        if (pair) {
            double2 wp = first ? wip : tw[((int64_t)k1p * i2) % L];
            T[(int64_t)k1p * L2 + i2] = cmul(B[i2], cconj(wp));
        }
    }
}

__global__ void k_hist_icols(DevPlan P, const double2* __restrict__ T) {
    extern __shared__ double2 sm[];
    double2* twN = sm + P.L1;
    int i2 = blockIdx.x;
    int logL1 = 31 - __clz(P.L1);
    const double2* tw = (const double2*)P.twiddle;
    for (int k1 = threadIdx.x; k1 < P.L1; k1 += blockDim.x) {
        double2 v = T[(int64_t)k1 * P.L2 + i2];
        double2 t = k1 < P.L1 / 2 ? tw[k1 * (P.L / P.L1)] : make_double2(0.0, 0.0);
        sm[__brev(k1) >> (32 - logL1)] = v;
        if (k1 < P.L1 / 2) twN[k1] = make_double2(t.x, -t.y);
    }
    __syncthreads();
    fft_line(sm, twN, P.L1, logL1);
    double2* grid = (double2*)P.grid;
    for (int i1 = threadIdx.x; i1 < P.L1; i1 += blockDim.x) grid[i2 + (int64_t)P.L2 * i1] = sm[i1];
}

}  // namespace wave1d
