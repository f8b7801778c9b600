// Standalone NUFFTs of the history part (Sec. 3.1) on fixed points: the type-1 transform
// S_k = (1/2 pi) sum_j c_j e^{+i k x_j}, k = 0..K (eq. densco), and the type-2 transform
// u_j = sum_{|k| <= K} alpha_k e^{-i k x_j} with alpha_{-k} = conj(alpha_k) (eq. historySol1), each
// split into its spreading (A1) or interpolation (A6) pass and the FFT, with the same Kaiser-Bessel
// kernel, fine grid and deconvolution as the time-step plan.  A plan may hold many point sets
// (instances) with the same K; one launch per pass covers all of them.
//
// Two precisions:
//   FP64   kernel weights precomputed (w per point) and streamed from HBM.  Relative accuracy set
//          by tol, like the time-step plan.
//   mixed  each tap's kernel a Chebyshev series in the point's offset within its first cell
//          (fitted on the host to about 2e-7 of the kernel's peak); spreading by per-cell
//          Chebyshev moments and interpolation by per-cell Chebyshev sums of the grid, in FP32
//          with the dominant terms compensated; the FFT and the deconvolution stay FP64.  GB300
//          runs FP32 about 60 times faster than FP64, so these passes read little more than the
//          points' cells, offsets and values.
// Points are kept in an internal order sorted by first grid cell, instance by instance
// (wave1d_nufft_perm gives it).  Spreading: each instance's grid is cut into cell ranges, one
// block per range writes its grid reals complete (recomputing the sums of the w - 1 cells before
// the range), so clustered points, with hundreds per cell, spread over many blocks and lanes.
// Interpolation: blocks of consecutive points.  Neither uses atomics: the results do not depend
// on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "nufft_host.h"
#include "nufft_units.cuh"
#include "device_common.cuh"
#include "../../include/wave1d.h"

namespace wave1d {
__global__ void k_fft_cols(const double2*, double2*, const double2*, int, int, int, int, int);
__global__ void k_fft_rows(const double2*, double2*, const double2*, int, int, int, int, int);
}  // namespace wave1d

using namespace wave1d;

namespace {

constexpr double kPiN = 3.14159265358979323846264338327950288;
constexpr int kMaxDegree = 16;      // polynomial degree limit of the mixed-precision kernel

thread_local std::string g_nu_error;

int nfail(int code, const std::string& msg) {
    g_nu_error = msg;
    return code;
}

// ---------------------------------------------------------------------------------------------
// Moving between FP64 and FP32 with integer operations on the IEEE-754 bit patterns.  On this GPU
// the FP64 pipe, conversions included, issues about 60 times slower than FP32, so the mixed passes
// convert each value with a few integer operations instead.
// ---------------------------------------------------------------------------------------------
// double -> float, rounded to nearest (ties away from zero); magnitudes below 2^-126 give a signed
// zero, magnitudes above the float range a signed infinity
__device__ __forceinline__ float nu_f64_to_f32(double d) {
    unsigned hw = (unsigned)__double2hiint(d);
    const unsigned lw = (unsigned)__double2loint(d);
    const unsigned lr = lw + 0x10000000u;                 // half a unit of the 29 dropped bits
    hw += lr < lw ? 1u : 0u;                              // a carry may step the exponent: still exact
    const unsigned s = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7ffu) - 896;       // biased float exponent
    const unsigned b = s | ((unsigned)e << 23) | ((hw & 0xfffffu) << 3) | (lr >> 29);
    return __uint_as_float(e <= 0 ? s : (e >= 255 ? (s | 0x7f800000u) : b));
}
// float -> double, exact for zero and normal floats (subnormals give a signed zero)
__device__ __forceinline__ double nu_f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu, s = b & 0x80000000u;
    const unsigned hw = e == 0u ? s : (e == 255u ? (s | 0x7ff00000u) : (s | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)));
    const unsigned lw = (e == 0u || e == 255u) ? 0u : (b << 29);
    return __hiloint2double((int)hw, (int)lw);
}

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void nu_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (sh, sl) += (ph, pl)
__device__ __forceinline__ void nu_pair_add(float& sh, float& sl, float ph, float pl) {
    float s, t;
    nu_two_sum(sh, ph, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, pl));
}

// Mixed-precision kernel: tap t (0 <= t < w) of a point with offset variable y in [-1, 1] has the
// value psi_t(y) = sum_d a[t][d] T_d(y), a Chebyshev series of degree D fitted on the host (well
// conditioned: sum_d |a[t][d]| stays near max psi_t, so FP32 evaluation loses little).  The
// kernel is even, so psi_{w-1-t}(y) = psi_t(-y) and a[w-1-t][d] = (-1)^d a[t][d]: the host fits
// the first half of the taps and mirrors them.  The table is a kernel parameter, so the unrolled
// FMAs take their coefficients straight from the constant bank.
struct NuPoly {
    float c[16][kMaxDegree + 1];
};
template <int D>
struct NuCheb {                    // T_0(y) .. T_D(y) by the three-term recurrence
    float T[D + 1];
    __device__ __forceinline__ explicit NuCheb(float y) {
        const float y2 = __fadd_rn(y, y);
        T[0] = 1.f;
        T[1] = y;
#pragma unroll
        for (int d = 2; d <= D; d++) T[d] = __fmaf_rn(y2, T[d - 1], -T[d - 2]);
    }
};
// all w kernel values of a point: even and odd parts of the first half, mirrored
template <int W, int D>
__device__ __forceinline__ void nu_taps(const NuPoly& P, const NuCheb<D>& ch, float (&psi)[W]) {
#pragma unroll
    for (int t = 0; t < (W + 1) / 2; t++) {
        float e = P.c[t][0], o = __fmul_rn(P.c[t][1], ch.T[1]);
#pragma unroll
        for (int d = 2; d <= D; d += 2) e = __fmaf_rn(P.c[t][d], ch.T[d], e);
#pragma unroll
        for (int d = 3; d <= D; d += 2) o = __fmaf_rn(P.c[t][d], ch.T[d], o);
        psi[t] = __fadd_rn(e, o);
        if (W - 1 - t != t) psi[W - 1 - t] = __fsub_rn(e, o);
    }
}

// ---------------------------------------------------------------------------------------------
// Spreading (A1).  The points are sorted by first cell; the grid is cut into cell ranges, each
// range handled by one block that writes its grid reals complete (below).  No atomics: the result
// does not depend on scheduling, and a dense cluster (hundreds of points per cell) spreads over
// many ranges and lanes.
// ---------------------------------------------------------------------------------------------

// Mixed precision by Chebyshev moments.  With psi_t(y) = sum_d a[t][d] T_d(y),
//   G[g] = sum_t sum_{q: i0_q = g - t} c_q psi_t(y_q) = sum_t sum_d a[t][d] M_d(g - t),
//   M_d(f) = sum_{q: i0_q = f} c_q T_d(y_q),
// so a point costs D + 1 FMAs (its moments) and each grid real w (D + 1) multiply-adds.
//
// Work split: the grid is tiled by cell ranges [c0, c0 + nc) (at most kRangeCells cells, and at
// most kRangePoints points counting the w - 1 cells before the range, the halo).  A block takes a
// range: it stages the (c, y) of the points whose first cell lies in [c0 - w + 1, c0 + nc) in
// shared memory (one or two slices of the sorted points: the halo of the first range wraps round
// the periodic box), gives each of those nc + w - 1 cells a group of G lanes that accumulate the
// cell's moments (a fixed shuffle tree closes each group), and then writes every grid real of its
// range complete.  The halo cells' moments are computed twice, by this block and by the
// previous one; in exchange no block depends on another (no partials, atomics or second pass),
// each grid real is written once, and the result does not depend on scheduling.  A range whose
// points exceed kStage (a cell holding thousands of points) reads them from global memory.
// M_0 and the d = 0 terms are compensated FP32 pairs (they carry the magnitude); the higher
// moments cancel over a cell and carry small coefficients, so they are plain FP32.
constexpr int kStage = 2048;        // staging capacity (points) of a range
constexpr int kRangePoints = 2048;  // points a range is cut at, halo included (one cell may exceed it)
constexpr int kRangeCells = 240;    // cells of a mixed range (w - 1 halo cells more fit one thread each)
constexpr int kRangePoints64 = 4096;  // FP64: its halo costs FP64 FMAs, so fewer, larger ranges
constexpr int kEmptyCells = 8192;   // cells of a range no point reaches (zeros only)
template <int W, int D>
__global__ void __launch_bounds__(kUnitThreads) k_nu_spread_mixed(const NuRange* __restrict__ ranges,
                                                                  const int32_t* __restrict__ runs,
                                                                  const double* __restrict__ c,
                                                                  const float* __restrict__ soff, const NuPoly P,
                                                                  double* __restrict__ grid) {
    constexpr int R = (D + 2 + 3) / 4 * 4;            // moment row: M_0 (hi, lo), M_1 .. M_D, padded to float4
    constexpr int kPer = kStage / kUnitThreads;
    __shared__ int rp[kRangeCells + 16 + 1];
    __shared__ float2 cy[kStage];
    __shared__ __align__(16) float mo[kRangeCells + 16][R];
    const NuRange u = ranges[blockIdx.x];
    const int nr = u.nc + W - 1, np = u.na + u.nb;
    if (np == 0) {                                    // no point reaches the range: zeros
        for (int l = threadIdx.x; l < u.nc; l += kUnitThreads) grid[u.c0 + l] = 0.0;
        return;
    }
    const bool staged = np <= kStage;
    if ((int)threadIdx.x <= nr) rp[threadIdx.x] = __ldg(runs + u.roff + threadIdx.x);
    if (staged) {
        double cd[kPer];
        float sv[kPer];
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int q = (int)threadIdx.x + i * kUnitThreads;
            if (q < np) {
                const int j = q < u.na ? u.a0 + q : u.b0 + (q - u.na);
                cd[i] = __ldcs(c + j);
                sv[i] = __ldcs(soff + j);
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int q = (int)threadIdx.x + i * kUnitThreads;
            if (q < np) cy[q] = make_float2(nu_f64_to_f32(cd[i]), __fmaf_rn(2.f, sv[i], -1.f));
        }
    }
    __syncthreads();
    const int G = 1 << u.lg, f = (int)threadIdx.x >> u.lg, gl = (int)threadIdx.x & (G - 1);
    float m[D + 1];
#pragma unroll
    for (int d = 0; d <= D; d++) m[d] = 0.f;
    if (f < nr) {
        const int q1 = rp[f + 1];
        for (int q = rp[f] + gl; q < q1; q += G) {
            float2 v;
            if (staged) {
                v = cy[q];
            } else {
                const int j = q < u.na ? u.a0 + q : u.b0 + (q - u.na);
                v = make_float2(nu_f64_to_f32(__ldcs(c + j)), __fmaf_rn(2.f, __ldcs(soff + j), -1.f));
            }
            const NuCheb<D> ch(v.y);
            m[0] = __fadd_rn(m[0], v.x);
#pragma unroll
            for (int d = 1; d <= D; d++) m[d] = __fmaf_rn(ch.T[d], v.x, m[d]);
        }
    }
    float m0l = 0.f;
    for (int o = G >> 1; o > 0; o >>= 1) {
        nu_pair_add(m[0], m0l, __shfl_xor_sync(0xffffffffu, m[0], o), __shfl_xor_sync(0xffffffffu, m0l, o));
#pragma unroll
        for (int d = 1; d <= D; d++) m[d] = __fadd_rn(m[d], __shfl_xor_sync(0xffffffffu, m[d], o));
    }
    if (gl == 0 && f < nr) {
        mo[f][0] = m[0];
        mo[f][1] = m0l;
#pragma unroll
        for (int d = 1; d <= D; d++) mo[f][d + 1] = m[d];
    }
    __syncthreads();
    if ((int)threadIdx.x < u.nc && rp[threadIdx.x + W] == rp[threadIdx.x]) {
        grid[u.c0 + threadIdx.x] = 0.0;               // none of the w cells feeding it holds a point
    } else if ((int)threadIdx.x < u.nc) {
        // grid real c0 + l takes tap t of cell c0 + l - t, i.e. run (l + w - 1) - t
        const int l = threadIdx.x;
        float h = 0.f, lo = 0.f, r = 0.f;
#pragma unroll
        for (int t = 0; t < W; t++) {
            float mf[R];
#pragma unroll
            for (int k = 0; k < R; k += 4)
                *reinterpret_cast<float4*>(mf + k) = *reinterpret_cast<const float4*>(&mo[l + W - 1 - t][k]);
            const float p = __fmul_rn(P.c[t][0], mf[0]);
            const float e = __fmaf_rn(P.c[t][0], mf[1], __fmaf_rn(P.c[t][0], mf[0], -p));
            nu_pair_add(h, lo, p, e);
#pragma unroll
            for (int d = 1; d <= D; d++) r = __fmaf_rn(P.c[t][d], mf[d + 1], r);
        }
        nu_pair_add(h, lo, r, 0.f);
        grid[u.c0 + l] = nu_f32_to_f64(h) + nu_f32_to_f64(lo);
    }
}

// FP64 spreading on the same cell ranges, one block per range (spread64_unit, nufft_units.cuh).
// Like the mixed pass, no block depends on another.
template <int W>
__global__ void __launch_bounds__(kUnitThreads) k_nu_spread64(const NuRange* __restrict__ ranges,
                                                              const int32_t* __restrict__ runs,
                                                              const double* __restrict__ c,
                                                              const double* __restrict__ ker,
                                                              double* __restrict__ grid) {
    __shared__ int rp[kSpread64Runs];
    __shared__ double seg[kRangeCells64 + 16][W];
    spread64_unit<W>(ranges[blockIdx.x], runs, c, ker, grid, seg, rp);
}

// type-1 post-processing: S_k from the half-length FFT Z (E, O split) with the deconvolution
// factors: S_k = f0 E_k + (f1 + i f2) O_k
__global__ void k_nu_post1(const double2* __restrict__ Z, double* __restrict__ S, const double* __restrict__ modefac,
                           int K, int L) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > K) return;
    const double2 zk = Z[k], zm = Z[k == 0 ? 0 : L - k];
    const double* f = modefac + 8 * (int64_t)k;
    const double2 E = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    const double2 D = make_double2(0.5 * (zk.x - zm.x), 0.5 * (zk.y + zm.y));
    const double2 O = make_double2(D.y, -D.x);
    const double2 s = cadd(make_double2(f[0] * E.x, f[0] * E.y), cmul(make_double2(f[1], f[2]), O));
    S[2 * k] = s.x;
    S[2 * k + 1] = s.y;
}

// type-2 spectrum for the inverse real FFT: Zs[k] = alpha_k (f3 + i f4), Zs[L - k] =
// conj(alpha_k) (f5 + i f6), zero where no mode lands
__global__ void k_nu_pre2(const double* __restrict__ alpha, double2* __restrict__ Zs, const double* __restrict__ modefac,
                          int K, int L) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L; idx += gridDim.x * blockDim.x) {
        double2 z = make_double2(0.0, 0.0);
        if (idx <= K) {
            const double* f = modefac + 8 * (int64_t)idx;
            z = cmul(make_double2(alpha[2 * idx], alpha[2 * idx + 1]), make_double2(f[3], f[4]));
        } else if (idx >= L - K) {
            const int k = L - idx;
            const double* f = modefac + 8 * (int64_t)k;
            z = cmul(make_double2(alpha[2 * k], -alpha[2 * k + 1]), make_double2(f[5], f[6]));
        }
        Zs[idx] = z;
    }
}

// FP64 interpolation, tiles of kInterpTile consecutive points (interp64_unit, nufft_units.cuh).
__global__ void __launch_bounds__(kInterpTile) k_nu_interp64(const double* __restrict__ grid, double* __restrict__ u,
                                                             const int32_t* __restrict__ i0,
                                                             const double* __restrict__ ker, int64_t M, int w, int nf) {
    __shared__ double ks[kInterpTile * 16];
    const int64_t tiles = (M + kInterpTile - 1) / kInterpTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) interp64_unit(t, grid, u, i0, ker, M, w, nf, ks);
}

// mixed interpolation (A6).  With psi_t(y) = sum_d a[t][d] T_d(y),
//   u_j = sum_t psi_t(y_j) G[i0_j + t] = sum_d T_d(y_j) H_d(i0_j),  H_d(i) = sum_t a[t][d] G[i + t],
// and H depends only on the first cell.  A block takes 1024 consecutive points (sorted by first
// cell, four per thread), converts the grid cells they reach to FP32 in shared memory, forms H
// for each of their first cells (W (D + 1) FMAs per cell), and then each point costs D + 1 FMAs.
// FP32 throughout (rounding of the order of the kernel's fit, below the requested tolerance).  A
// block whose points start in more than kHCells cells evaluates the taps per point instead.
constexpr int kHCells = 512;
constexpr int kInterpPer = 4;
template <int W, int D>
__global__ void __launch_bounds__(256) k_nu_interp_mixed(const double* __restrict__ grid, double* __restrict__ u,
                                                         const int32_t* __restrict__ first,
                                                         const float* __restrict__ soff, const NuPoly P, int64_t M,
                                                         int nf) {
    constexpr int R = (D + 1 + 3) / 4 * 4;            // H row, padded to float4
    __shared__ float gs[kHCells + 16];
    __shared__ __align__(16) float H[kHCells * R];
    __shared__ int fr[2];
    const int64_t base = (int64_t)blockIdx.x * (256 * kInterpPer);
    const int64_t last = M - 1 < base + 256 * kInterpPer - 1 ? M - 1 : base + 256 * kInterpPer - 1;
    int a[kInterpPer];
    float y[kInterpPer];
#pragma unroll
    for (int i = 0; i < kInterpPer; i++) {
        const int64_t j = base + threadIdx.x + i * 256;
        a[i] = j <= last ? __ldg(first + j) : 0;
        y[i] = j <= last ? __fmaf_rn(2.f, __ldcs(soff + j), -1.f) : 0.f;
        if (j == base) fr[0] = a[i];
        if (j == last) fr[1] = a[i];
    }
    __syncthreads();
    // cells are instance x nf + cell (nf a power of two): a block within one instance wraps inside
    // it; a block that straddles two instances takes the per-point path
    const int c0 = fr[0], ncell = fr[1] - c0 + 1, gbase = c0 & ~(nf - 1);
    const bool fits = ncell <= kHCells && (fr[1] & ~(nf - 1)) == gbase;   // the same in every thread
    if (fits) {
        for (int l = threadIdx.x; l < ncell + W - 1; l += 256)
            gs[l] = nu_f64_to_f32(__ldg(grid + (gbase | ((c0 + l) & (nf - 1)))));
        __syncthreads();
        for (int l = threadIdx.x; l < ncell; l += 256) {
            float g[W];
#pragma unroll
            for (int t = 0; t < W; t++) g[t] = gs[l + t];
#pragma unroll
            for (int d = 0; d <= D; d++) {
                float h = __fmul_rn(P.c[0][d], g[0]);
#pragma unroll
                for (int t = 1; t < W; t++) h = __fmaf_rn(P.c[t][d], g[t], h);
                H[l * R + d] = h;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kInterpPer; i++) {
        const int64_t j = base + threadIdx.x + i * 256;
        if (j > last) break;
        const NuCheb<D> ch(y[i]);
        float acc;
        if (fits) {
            float h[R];
#pragma unroll
            for (int k = 0; k < R; k += 4) *reinterpret_cast<float4*>(h + k) = *reinterpret_cast<const float4*>(H + (a[i] - c0) * R + k);
            acc = h[0];
#pragma unroll
            for (int d = 1; d <= D; d++) acc = __fmaf_rn(ch.T[d], h[d], acc);
        } else {
            float psi[W];
            nu_taps<W, D>(P, ch, psi);
            acc = 0.f;
            const int pb = a[i] & ~(nf - 1);
#pragma unroll
            for (int t = 0; t < W; t++)
                acc = __fmaf_rn(psi[t], nu_f64_to_f32(__ldg(grid + (pb | ((a[i] + t) & (nf - 1))))), acc);
        }
        __stcs(u + j, nu_f32_to_f64(acc));
    }
}

// compile-time kernel widths and polynomial degrees: FP64 takes w = 4..16; mixed precision
// (tol >= 1e-6) takes w = 4..7 with degrees 6, 8 or 10
constexpr int kMixedMaxW = 7;
template <int W, typename F>
bool nu_try_w(int w, F& f) {
    if (w != W) return false;
    f(std::integral_constant<int, W>{});
    return true;
}
template <typename F>
bool nu_with_w(int w, F&& f) {
    return nu_try_w<4>(w, f) || nu_try_w<5>(w, f) || nu_try_w<6>(w, f) || nu_try_w<7>(w, f) ||
           nu_try_w<8>(w, f) || nu_try_w<9>(w, f) || nu_try_w<10>(w, f) || nu_try_w<11>(w, f) ||
           nu_try_w<12>(w, f) || nu_try_w<13>(w, f) || nu_try_w<14>(w, f) || nu_try_w<15>(w, f) ||
           nu_try_w<16>(w, f);
}
template <typename F>
bool nu_with_mixed(int w, int D, F&& f) {
    auto wd = [&](auto wc, auto dc) {
        if (wc.value != w || dc.value != D) return false;
        f(wc, dc);
        return true;
    };
    using I4 = std::integral_constant<int, 4>;
    using I5 = std::integral_constant<int, 5>;
    using I6 = std::integral_constant<int, 6>;
    using I7 = std::integral_constant<int, 7>;
    using I8 = std::integral_constant<int, 8>;
    using I10 = std::integral_constant<int, 10>;
    return wd(I4{}, I6{}) || wd(I4{}, I8{}) || wd(I4{}, I10{}) || wd(I5{}, I6{}) || wd(I5{}, I8{}) ||
           wd(I5{}, I10{}) || wd(I6{}, I6{}) || wd(I6{}, I8{}) || wd(I6{}, I10{}) || wd(I7{}, I6{}) ||
           wd(I7{}, I8{}) || wd(I7{}, I10{});
}

int ilog2n(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

}  // namespace

struct wave1d_nufft_s {
    int device = 0;
    int precision = 0;
    int64_t M = 0;                   // points over all instances
    int B = 1;                       // instances (each with its own grid of nf reals)
    Params P{};
    int D = 0;                       // polynomial degree (mixed)
    double kernel_err = 0.0;         // max |Chebyshev series (FP32) - kernel| over the taps (mixed)
    cudaStream_t stream = nullptr;
    std::vector<int64_t> perm;       // internal point i -> caller index
    std::vector<void*> allocs;
    // points (internal order): first cell, offset in it (mixed), kernel weights (FP64)
    int32_t* first = nullptr;
    float* soff = nullptr;
    NuPoly poly{};                   // tap polynomials (mixed), passed to the kernels by value
    double* ker = nullptr;
    // spreading ranges (cell ranges tiling every instance's grid) and their run tables
    NuRange* ranges = nullptr;
    int64_t nunits = 0;              // ranges
    int32_t* runs = nullptr;
    int range_cells = 0, range_points = 0;   // the caps the ranges were cut with
    std::vector<int32_t> i0_host;    // points' first cells (sorted within each instance), for re-cutting
    std::vector<int64_t> off_host;   // instance offsets
    // FFT and deconvolution
    double *grid = nullptr, *work = nullptr, *spec = nullptr, *spec2 = nullptr, *twiddle = nullptr,
           *modefac = nullptr;
};

namespace {

template <typename T>
int nu_upload(wave1d_nufft_t h, const std::vector<T>& v, T** out) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nfail(WAVE1D_ENOMEM, "cudaMalloc failed");
    h->allocs.push_back(p);
    if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return nfail(WAVE1D_ECUDA, "cudaMemcpy failed");
    *out = (T*)p;
    return WAVE1D_OK;
}

template <typename T>
int nu_alloc(wave1d_nufft_t h, size_t count, T** out) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess)
        return nfail(WAVE1D_ENOMEM, "cudaMalloc failed");
    h->allocs.push_back(p);
    *out = (T*)p;
    return WAVE1D_OK;
}

}  // namespace

namespace wave1d {
int nufft_dev64(wave1d_nufft_t h, NuDev64& out) {
    if (!h || h->precision != 0) return WAVE1D_EINVAL;
    out.ranges = h->ranges;
    out.runs = h->runs;
    out.nunits = h->nunits;
    out.ker = h->ker;
    out.i0 = h->first;
    out.M = h->M;
    out.w = h->P.nufft_w;
    out.nf = h->P.nf;
    return WAVE1D_OK;
}
}  // namespace wave1d

extern "C" {

int wave1d_nufft_plan(const double* x, int64_t M, int K, double tol, int precision, void* stream,
                      wave1d_nufft_t* out) {
    if (!out) return nfail(WAVE1D_EINVAL, "out is NULL");
    *out = nullptr;
    const int64_t off[2] = {0, M};
    return wave1d_nufft_plan_many(x, off, 1, K, tol, precision, stream, out);
}

int wave1d_nufft_plan_many(const double* x, const int64_t* offsets, int n_inst, int K, double tol, int precision,
                           void* stream, wave1d_nufft_t* out) {
    if (!out) return nfail(WAVE1D_EINVAL, "out is NULL");
    *out = nullptr;
    if (!x || !offsets || n_inst < 1 || K < 1 || !(tol > 0.0 && tol < 0.1) || (precision != 0 && precision != 1))
        return nfail(WAVE1D_EINVAL, "need x, offsets, n_instances >= 1, K >= 1, 0 < tol < 0.1, precision 0 or 1");
    if (offsets[0] != 0) return nfail(WAVE1D_EINVAL, "offsets[0] must be 0");
    for (int b = 0; b < n_inst; b++)
        if (offsets[b + 1] <= offsets[b]) return nfail(WAVE1D_EINVAL, "every instance needs at least one point");
    const int64_t M = offsets[n_inst];
    if (M > INT32_MAX / 32) return nfail(WAVE1D_EINVAL, "at most 2^26 points in all");
    if (precision == 1 && tol < 1e-6) return nfail(WAVE1D_EINVAL, "mixed precision needs tol >= 1e-6");
    wave1d_nufft_t h = new (std::nothrow) wave1d_nufft_s();
    if (!h) return nfail(WAVE1D_ENOMEM, "host allocation");
    auto cleanup = [&](int code) {
        wave1d_nufft_destroy(h);
        return code;
    };
    h->precision = precision;
    h->M = M;
    h->B = n_inst;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) return cleanup(nfail(WAVE1D_ECUDA, "no CUDA device"));
    Params& P = h->P;
    nufft_grid(P, K, tol, 0);
    if (P.L2 > 1024) return cleanup(nfail(WAVE1D_EUNSUPPORTED, "fine grid too large for this build (nf > 2^21)"));
    if ((int64_t)n_inst * P.nf > INT32_MAX / 2) return cleanup(nfail(WAVE1D_EINVAL, "instances x fine grid above 2^30"));
    const int w = P.nufft_w, nf = P.nf;
    // positions wrapped into [-pi, pi), kernel weights, internal order: instance by instance, each
    // sorted by first cell
    std::vector<double> xw(M);
    for (int64_t j = 0; j < M; j++) {
        double v = x[j];
        if (!std::isfinite(v)) return cleanup(nfail(WAVE1D_EINVAL, "non-finite position"));
        v = std::fmod(v + kPiN, 2.0 * kPiN);
        if (v < 0) v += 2.0 * kPiN;
        v -= kPiN;
        if (v >= kPiN) v -= 2.0 * kPiN;
        xw[j] = v;
    }
    std::vector<int32_t> i0c;
    std::vector<double> kerc;
    spread_weights(P, xw, i0c, kerc);
    h->perm.resize(M);
    std::iota(h->perm.begin(), h->perm.end(), 0);
    for (int b = 0; b < n_inst; b++)
        std::stable_sort(h->perm.begin() + offsets[b], h->perm.begin() + offsets[b + 1], [&](int64_t p, int64_t q) {
            return i0c[p] != i0c[q] ? i0c[p] < i0c[q] : xw[p] < xw[q];
        });
    std::vector<int32_t> i0(M), gfirst(M);           // cell in the instance; instance x nf + cell
    std::vector<double> xs(M);
    for (int b = 0; b < n_inst; b++)
        for (int64_t i = offsets[b]; i < offsets[b + 1]; i++) {
            i0[i] = i0c[h->perm[i]];
            gfirst[i] = b * nf + i0[i];
            xs[i] = xw[h->perm[i]];
        }
    int rc;
    if (precision == 0) {
        std::vector<double> ker((size_t)M * w);
        for (int64_t i = 0; i < M; i++)
            std::memcpy(&ker[(size_t)i * w], &kerc[(size_t)h->perm[i] * w], sizeof(double) * w);
        if ((rc = nu_upload(h, ker, &h->ker))) return cleanup(rc);
    } else {
        // offsets s = first - u + w/2 in [0, 1), y = 2 s - 1; tap t's kernel as a polynomial in y
        std::vector<float> soff(M);
        for (int64_t i = 0; i < M; i++) {
            const double u = (xs[i] + kPiN) / P.h_f;
            const double fst = std::ceil(u - 0.5 * w);
            soff[i] = (float)(fst - u + 0.5 * w);
        }
        const int ns = 96;
        std::vector<double> ys(ns);
        for (int i = 0; i < ns; i++) ys[i] = std::cos(kPiN * (i + 0.5) / ns);
        const double inv_i0b = 1.0 / std::cyl_bessel_i(0.0, P.kb_beta);
        auto kernel = [&](double y, int t) {
            double s = 0.5 * (y + 1.0);
            double z = (s + t - 0.5 * w) * 2.0 / w;
            double r = 1.0 - z * z;
            return r > 0.0 ? std::cyl_bessel_i(0.0, P.kb_beta * std::sqrt(r)) * inv_i0b : 0.0;
        };
        // Chebyshev series of degree 6, 8 or 10 (the ones the kernels are built for): the first
        // within max(3e-7, tol / 5) of the kernel (FP32 evaluation alone errs by about 1.7e-7), checked
        // in FP32 in the device's order.  Taps
        // t < w/2 are fitted (coefficients from the discrete Chebyshev transform at ns nodes, a
        // near-minimax truncation); tap w-1-t mirrors t, and the middle tap of an odd w keeps only
        // its even terms.
        if (w > kMixedMaxW) return cleanup(nfail(WAVE1D_EINVAL, "mixed precision: kernel width above 7"));
        const double fit_tol = std::max(3e-7, tol / 5);
        int D = 6;
        double err = 1.0;
        for (;; D += 2) {
            std::memset(&h->poly, 0, sizeof(h->poly));
            for (int t = 0; t < (w + 1) / 2; t++) {
                for (int d = 0; d <= D; d++) {
                    double acc = 0.0;
                    for (int i = 0; i < ns; i++) acc += kernel(ys[i], t) * std::cos(d * kPiN * (i + 0.5) / ns);
                    double ad = (d == 0 ? 1.0 : 2.0) * acc / ns;
                    if (2 * t + 1 == w && d % 2 == 1) ad = 0.0;
                    h->poly.c[t][d] = (float)ad;
                    h->poly.c[w - 1 - t][d] = (float)(d % 2 ? -ad : ad);
                }
            }
            // interior points: at y = -1 and +1 an end tap touches the support edge, where the
            // kernel drops from 1/I0(beta) to 0 (a jump of the kernel itself, not of the fit)
            err = 0.0;
            for (int i = 1; i < 400; i++) {
                const float y = (float)(-1.0 + 2.0 * i / 400.0);
                float T[kMaxDegree + 1];
                T[0] = 1.f;
                T[1] = y;
                for (int d = 2; d <= D; d++) T[d] = std::fma(y + y, T[d - 1], -T[d - 2]);
                for (int t = 0; t < (w + 1) / 2; t++) {
                    float e = h->poly.c[t][0], o = h->poly.c[t][1] * T[1];
                    for (int d = 2; d <= D; d += 2) e = std::fma(h->poly.c[t][d], T[d], e);
                    for (int d = 3; d <= D; d += 2) o = std::fma(h->poly.c[t][d], T[d], o);
                    err = std::max(err, std::fabs((double)(e + o) - kernel((double)y, t)));
                    err = std::max(err, std::fabs((double)(e - o) - kernel((double)y, w - 1 - t)));
                }
            }
            if (err < fit_tol || D == 10) break;
        }
        h->D = D;
        h->kernel_err = err;
        if ((rc = nu_upload(h, soff, &h->soff))) return cleanup(rc);
    }
    {
        std::vector<NuRange> ranges;
        std::vector<int32_t> runs;
        nufft_ranges(i0, offsets, n_inst, nf, w, precision == 1 ? kRangeCells : kRangeCells64,
                     precision == 1 ? kRangePoints : kRangePoints64, kEmptyCells, kUnitThreads, ranges, runs);
        h->nunits = (int64_t)ranges.size();
        h->range_cells = precision == 1 ? kRangeCells : kRangeCells64;
        h->range_points = precision == 1 ? kRangePoints : kRangePoints64;
        h->i0_host = i0;
        h->off_host.assign(offsets, offsets + n_inst + 1);
        if ((rc = nu_upload(h, ranges, &h->ranges)) || (rc = nu_upload(h, runs, &h->runs)) ||
            (rc = nu_upload(h, gfirst, &h->first)))
            return cleanup(rc);
    }
    std::vector<double> d1, d2, mf, tw((size_t)P.L * 2);
    nufft_factors(P, d1, d2, mf);
    for (int j = 0; j < P.L; j++) {
        double ang = 2.0 * kPiN * (double)j / (double)P.L;
        tw[2 * j] = std::cos(ang);
        tw[2 * j + 1] = std::sin(ang);
    }
    if ((rc = nu_upload(h, mf, &h->modefac)) || (rc = nu_upload(h, tw, &h->twiddle)) ||
        (rc = nu_alloc(h, (size_t)n_inst * nf, &h->grid)) || (rc = nu_alloc(h, (size_t)nf, &h->work)) ||
        (rc = nu_alloc(h, (size_t)nf, &h->spec)) || (rc = nu_alloc(h, (size_t)nf, &h->spec2)))
        return cleanup(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return cleanup(nfail(WAVE1D_ECUDA, "upload failed"));
    *out = h;
    return WAVE1D_OK;
}

int wave1d_nufft_info(wave1d_nufft_t h, int* nf, int* w, int* degree, double* kernel_err) {
    if (!h) return nfail(WAVE1D_EINVAL, "plan is NULL");
    if (nf) *nf = h->P.nf;
    if (w) *w = h->P.nufft_w;
    if (degree) *degree = h->D;
    if (kernel_err) *kernel_err = h->kernel_err;
    return WAVE1D_OK;
}

int wave1d_nufft_perm(wave1d_nufft_t h, int64_t* perm) {
    if (!h || !perm) return nfail(WAVE1D_EINVAL, "bad arguments");
    std::memcpy(perm, h->perm.data(), sizeof(int64_t) * h->M);
    return WAVE1D_OK;
}

int wave1d_nufft_spread(wave1d_nufft_t h, const double* c, double* grid) {
    if (!h || !c || !grid) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    const int w = h->P.nufft_w;
    const unsigned nu = (unsigned)h->nunits;
    bool ok;
    if (h->precision == 0) {
        ok = nu_with_w(w, [&](auto wc) {
            k_nu_spread64<decltype(wc)::value><<<nu, kUnitThreads, 0, h->stream>>>(h->ranges, h->runs, c, h->ker,
                                                                                    grid);
        });
    } else {
        ok = nu_with_mixed(w, h->D, [&](auto wc, auto dc) {
            k_nu_spread_mixed<decltype(wc)::value, decltype(dc)::value><<<nu, kUnitThreads, 0, h->stream>>>(
                h->ranges, h->runs, c, h->soff, h->poly, grid);
        });
    }
    if (!ok) return nfail(WAVE1D_EUNSUPPORTED, "kernel width / degree not built");
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "spread launch failed");
}

int wave1d_nufft_interp(wave1d_nufft_t h, const double* grid, double* u) {
    if (!h || !grid || !u) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    if (h->precision == 0) {
        k_nu_interp64<<<(unsigned)((h->M + kInterpTile - 1) / kInterpTile), kInterpTile, 0, h->stream>>>(
            grid, u, h->first, h->ker, h->M, h->P.nufft_w, h->P.nf);
    } else if (!nu_with_mixed(h->P.nufft_w, h->D, [&](auto wc, auto dc) {
                   const unsigned nb = (unsigned)((h->M + 256 * kInterpPer - 1) / (256 * kInterpPer));
                   k_nu_interp_mixed<decltype(wc)::value, decltype(dc)::value><<<nb, 256, 0, h->stream>>>(
                       grid, u, h->first, h->soff, h->poly, h->M, h->P.nf);
               })) {
        return nfail(WAVE1D_EUNSUPPORTED, "kernel width / degree not built");
    }
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "interp launch failed");
}

int wave1d_nufft_type1(wave1d_nufft_t h, const double* c, double* S) {
    if (!h || !c || !S) return nfail(WAVE1D_EINVAL, "bad arguments");
    int rc = wave1d_nufft_spread(h, c, h->grid);
    if (rc) return rc;
    const Params& P = h->P;
    const int t1 = std::max(32, std::min(P.L1 / 2, 512)), t2 = std::max(32, std::min(P.L2 / 2, 512));
    for (int b = 0; b < h->B; b++) {              // the instances' FFTs one after another
        k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), h->stream>>>((const double2*)(h->grid + (size_t)b * P.nf),
                                                                  (double2*)h->work, (const double2*)h->twiddle, P.L,
                                                                  P.L1, P.L2, ilog2n(P.L1), +1);
        k_fft_rows<<<P.L1, t2, fft_smem_bytes(P.L2), h->stream>>>((const double2*)h->work, (double2*)h->spec,
                                                                  (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                                  ilog2n(P.L2), +1);
        k_nu_post1<<<(P.K + 1 + 127) / 128, 128, 0, h->stream>>>((const double2*)h->spec,
                                                                 S + (size_t)b * 2 * (P.K + 1), h->modefac, P.K, P.L);
    }
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "type-1 launch failed");
}

int wave1d_nufft_type2(wave1d_nufft_t h, const double* alpha, double* u) {
    if (!h || !alpha || !u) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    const Params& P = h->P;
    const int t1 = std::max(32, std::min(P.L1 / 2, 512)), t2 = std::max(32, std::min(P.L2 / 2, 512));
    for (int b = 0; b < h->B; b++) {
        k_nu_pre2<<<(P.L + 255) / 256, 256, 0, h->stream>>>(alpha + (size_t)b * 2 * (P.K + 1), (double2*)h->spec2,
                                                             h->modefac, P.K, P.L);
        k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), h->stream>>>((const double2*)h->spec2, (double2*)h->work,
                                                                  (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                                  ilog2n(P.L1), -1);
        k_fft_rows<<<P.L1, t2, fft_smem_bytes(P.L2), h->stream>>>((const double2*)h->work,
                                                                  (double2*)(h->grid + (size_t)b * P.nf),
                                                                  (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                                  ilog2n(P.L2), -1);
    }
    if (cudaGetLastError() != cudaSuccess) return nfail(WAVE1D_ECUDA, "type-2 launch failed");
    return wave1d_nufft_interp(h, h->grid, u);
}

int wave1d_nufft_destroy(wave1d_nufft_t h) {
    if (!h) return WAVE1D_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (void* a : h->allocs) cudaFree(a);
    delete h;
    return WAVE1D_OK;
}

// Picks the spreading work split (its tile width and bin size: the cells and points a range is cut
// at) for this plan's points by timing: each candidate pair of caps, at or below the kernels'
// shared-memory capacities, re-cuts the ranges from the points' first cells and is timed over
// `reps` spreads of c (after one untimed spread) with CUDA events on the plan's stream; the fastest
// stays.  The grid is overwritten.  Every candidate tiles the grids completely (the range builder
// is the plan's own), so results change only in rounding (the lanes per cell follow the ranges).
int wave1d_nufft_autotune(wave1d_nufft_t h, const double* c, double* grid, int reps, int* cells, int* points) {
    if (!h || !c || !grid || reps < 1) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    const bool mixed = h->precision == 1;
    const int cmax = mixed ? kRangeCells : kRangeCells64, pmax = mixed ? kRangePoints : kRangePoints64;
    const int cand_c[3] = {cmax / 4, cmax / 2, cmax}, cand_p[3] = {pmax / 4, pmax / 2, pmax};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return nfail(WAVE1D_ECUDA, "cudaEventCreate");
    float best = 0.f;
    NuRange* best_r = h->ranges;
    int32_t* best_runs = h->runs;
    int64_t best_n = h->nunits;
    int best_c = h->range_cells, best_p = h->range_points;
    int rc = WAVE1D_OK;
    bool first = true;
    for (int ci = 0; ci < 3 && rc == WAVE1D_OK; ci++)
        for (int pi = 0; pi < 3 && rc == WAVE1D_OK; pi++) {
            std::vector<NuRange> ranges;
            std::vector<int32_t> runs;
            nufft_ranges(h->i0_host, h->off_host.data(), h->B, h->P.nf, h->P.nufft_w, cand_c[ci], cand_p[pi],
                         kEmptyCells, kUnitThreads, ranges, runs);
            NuRange* r_dev;
            int32_t* runs_dev;
            if ((rc = nu_upload(h, ranges, &r_dev)) || (rc = nu_upload(h, runs, &runs_dev))) break;
            h->ranges = r_dev;
            h->runs = runs_dev;
            h->nunits = (int64_t)ranges.size();
            if ((rc = wave1d_nufft_spread(h, c, grid))) break;
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps && rc == WAVE1D_OK; r++) rc = wave1d_nufft_spread(h, c, grid);
            cudaEventRecord(e1, h->stream);
            if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
                if (!rc) rc = nfail(WAVE1D_ECUDA, "timing the spreading failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (first || ms < best) {
                first = false;
                best = ms;
                best_r = r_dev;
                best_runs = runs_dev;
                best_n = h->nunits;
                best_c = cand_c[ci];
                best_p = cand_p[pi];
            }
        }
    h->ranges = best_r;
    h->runs = best_runs;
    h->nunits = best_n;
    h->range_cells = best_c;
    h->range_points = best_p;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (cells) *cells = best_c;
    if (points) *points = best_p;
    return WAVE1D_OK;
}

const char* wave1d_nufft_strerror(void) { return g_nu_error.c_str(); }

}  // extern "C"
