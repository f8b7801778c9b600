// Standalone NUFFTs of the history part (Sec. 3.1) on a fixed set of points: the type-1 transform
// S_k = (1/2 pi) sum_j c_j e^{+i k x_j}, k = 0..K (eq. densco), and the type-2 transform
// u_j = sum_{|k| <= K} alpha_k e^{-i k x_j} with alpha_{-k} = conj(alpha_k) (eq. historySol1), each
// split into its spreading (A1) or interpolation (A6) pass and the FFT, with the same Kaiser-Bessel
// kernel, fine grid and deconvolution as the time-step plan.
//
// Two precisions:
//   FP64   kernel weights precomputed (w per point) and streamed from HBM.  Relative accuracy set
//          by tol, like the time-step plan.
//   mixed  kernel values computed on the fly in FP32 from per-tap polynomials in the point's
//          offset within its first cell (fitted on the host to about 1e-7 of the kernel's peak),
//          sums in compensated FP32 pairs; the FFT and the deconvolution stay FP64.  GB300 runs
//          FP32 about 60 times faster than FP64, so these passes read little more than the points'
//          cells, offsets and values.
// Points are kept in an internal order sorted by first grid cell (wave1d_nufft_perm gives it).
// Spreading works on units of consecutive points (products in shared memory, one warp per cell,
// then a per-cell combine of the units' partials), so clustered points, with hundreds per cell,
// spread over many warps; the interpolation is one thread per point.  Neither uses atomics: the
// results do not depend on scheduling.
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
// value sum_d c[t][d] y^d (degree D, fitted on the host).  The table is a kernel parameter, so
// the unrolled Horner steps take their coefficients straight from the constant bank.
struct NuPoly {
    float c[16][kMaxDegree + 1];
};
template <int D>
__device__ __forceinline__ float nu_psi(const float (&c)[kMaxDegree + 1], float y) {
    float r = c[D];
#pragma unroll
    for (int d = D - 1; d >= 0; d--) r = __fmaf_rn(r, y, c[d]);
    return r;
}

// ---------------------------------------------------------------------------------------------
// Spreading by units (A1).  The host cuts the sorted points into units of at most kUnitPoints
// consecutive points whose first cells lie within kUnitCells cells.  A block takes a unit: each
// thread forms its point's w products kernel x c in shared memory; then each cell the unit
// reaches (its first cells plus w - 1) gets a group of G lanes (G a power of two, as many as the
// block can give every cell, at most 32) that sum the cell's contributors in point order, lanes
// strided, then by a fixed shuffle tree; the group stores the unit's partial for the cell.  A
// second pass adds, per grid real, the partials of the units that reach it, in unit order.  No
// atomics: the result does not depend on scheduling, and a dense cluster (hundreds of points per
// cell) spreads over many units and lanes.
// ---------------------------------------------------------------------------------------------
constexpr int kUnitPoints = 256;
constexpr int kUnitCells = 64;
constexpr int kValStride = 17;       // shared-memory stride of a point's products (odd: no bank conflicts)

struct NuUnit {
    int32_t pa, np, ca, span;     // first point, points, first cell, cells reached (< kUnitCells + w)
    int32_t poff, pad0, pad1, pad2; // offset of its partials
};

// first index in [lo, hi) of the sorted f[] with value >= v
__device__ __forceinline__ int nu_lower(const int* f, int lo, int hi, int v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (f[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// cell ranges of a unit: cstart[l] = first point whose first cell is >= ca + l (l <= kUnitCells);
// the G-lane group size for `span` cells
__device__ __forceinline__ int nu_unit_cells(const NuUnit& u, const int* fl, int* cstart) {
    if (threadIdx.x <= kUnitCells) cstart[threadIdx.x] = nu_lower(fl, 0, u.np, u.ca + (int)threadIdx.x);
    int lg = 5;
    while (lg > 0 && (u.span << lg) > kUnitPoints) lg--;
    return lg;
}

template <int D>
__global__ void __launch_bounds__(kUnitPoints) k_nu_spread_mixed(const NuUnit* __restrict__ units,
                                                                 const double* __restrict__ c,
                                                                 const int32_t* __restrict__ first,
                                                                 const float* __restrict__ soff, const NuPoly P,
                                                                 int w, float2* __restrict__ partial) {
    __shared__ int fl[kUnitPoints];
    __shared__ int cstart[kUnitCells + 1];
    __shared__ float val[kUnitPoints * kValStride];
    const NuUnit u = units[blockIdx.x];
    const int p = threadIdx.x;
    if (p < u.np) {
        const int64_t j = (int64_t)u.pa + p;
        fl[p] = __ldg(first + j);
        const float cj = nu_f64_to_f32(__ldcs(c + j));
        const float y = __fmaf_rn(2.f, __ldcs(soff + j), -1.f);
#pragma unroll
        for (int t = 0; t < 16; t++)
            if (t < w) val[p * kValStride + t] = __fmul_rn(nu_psi<D>(P.c[t], y), cj);
    }
    __syncthreads();
    const int lg = nu_unit_cells(u, fl, cstart);
    __syncthreads();
    const int G = 1 << lg, grp = p >> lg, gl = p & (G - 1);
    float sh = 0.f, sl = 0.f;
    if (grp < u.span) {
        const int g = u.ca + grp;
        const int lo = cstart[grp - w + 1 > 0 ? grp - w + 1 : 0];
        const int hi = cstart[grp + 1 < kUnitCells ? grp + 1 : kUnitCells];
        for (int q = lo + gl; q < hi; q += G) nu_pair_add(sh, sl, val[q * kValStride + (g - fl[q])], 0.f);
    }
    for (int o = G >> 1; o > 0; o >>= 1)
        nu_pair_add(sh, sl, __shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o));
    if (gl == 0 && grp < u.span) partial[u.poff + grp] = make_float2(sh, sl);
}

__global__ void __launch_bounds__(kUnitPoints) k_nu_spread64(const NuUnit* __restrict__ units,
                                                             const double* __restrict__ c,
                                                             const int32_t* __restrict__ first,
                                                             const double* __restrict__ ker, int w,
                                                             double* __restrict__ partial) {
    __shared__ int fl[kUnitPoints];
    __shared__ int cstart[kUnitCells + 1];
    __shared__ double cs[kUnitPoints];
    __shared__ double kv[kUnitPoints * kValStride];
    const NuUnit u = units[blockIdx.x];
    const int p = threadIdx.x;
    if (p < u.np) {
        fl[p] = __ldg(first + u.pa + p);
        cs[p] = __ldcs(c + u.pa + p);
    }
    // the unit's weights are one contiguous run of np w doubles: read it coalesced
    const double* kr = ker + (int64_t)u.pa * w;
    for (int e = p; e < u.np * w; e += kUnitPoints) {
        const int q = e / w;
        kv[q * kValStride + (e - q * w)] = __ldcs(kr + e);
    }
    __syncthreads();
    const int lg = nu_unit_cells(u, fl, cstart);
    __syncthreads();
    const int G = 1 << lg, grp = p >> lg, gl = p & (G - 1);
    double a = 0.0;
    if (grp < u.span) {
        const int g = u.ca + grp;
        const int lo = cstart[grp - w + 1 > 0 ? grp - w + 1 : 0];
        const int hi = cstart[grp + 1 < kUnitCells ? grp + 1 : kUnitCells];
        for (int q = lo + gl; q < hi; q += G) a = fma(kv[q * kValStride + (g - fl[q])], cs[q], a);
    }
    for (int o = G >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (gl == 0 && grp < u.span) partial[u.poff + grp] = a;
}

// combine pass: grid real r = sum of the partials of the units that reach r, in unit order
__global__ void k_nu_combine64(const double* __restrict__ partial, const int32_t* __restrict__ cptr,
                               const int32_t* __restrict__ cent, double* __restrict__ grid, int nf) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int e = __ldg(cptr + r); e < __ldg(cptr + r + 1); e++) a += __ldg(partial + __ldg(cent + e));
        grid[r] = a;
    }
}
__global__ void k_nu_combine32(const float2* __restrict__ partial, const int32_t* __restrict__ cptr,
                               const int32_t* __restrict__ cent, double* __restrict__ grid, int nf) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += gridDim.x * blockDim.x) {
        float sh = 0.f, sl = 0.f;
        for (int e = __ldg(cptr + r); e < __ldg(cptr + r + 1); e++) {
            const float2 v = __ldg(partial + __ldg(cent + e));
            nu_pair_add(sh, sl, v.x, v.y);
        }
        grid[r] = nu_f32_to_f64(sh) + nu_f32_to_f64(sl);
    }
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

// FP64 interpolation: u_j = sum_t G[(i0_j + t) mod nf] ker[j][t].  A block takes 256 consecutive
// points; their weights (one contiguous run of 256 w doubles) are staged through shared memory
// with coalesced streaming loads, and all w grid loads of a point are issued before any is used.
constexpr int kInterpTile = 256;
__global__ void __launch_bounds__(kInterpTile) k_nu_interp64(const double* __restrict__ grid, double* __restrict__ u,
                                                             const int32_t* __restrict__ i0,
                                                             const double* __restrict__ ker, int64_t M, int w, int nf) {
    __shared__ double ks[kInterpTile * 16];
    for (int64_t base = (int64_t)blockIdx.x * kInterpTile; base < M; base += (int64_t)gridDim.x * kInterpTile) {
        const int np = (int)(M - base < kInterpTile ? M - base : kInterpTile);
        __syncthreads();
        const double* kr = ker + base * w;
        for (int e = threadIdx.x; e < np * w; e += kInterpTile) ks[e] = __ldcs(kr + e);
        __syncthreads();
        if (threadIdx.x < np) {
            const int64_t j = base + threadIdx.x;
            const int a = __ldg(i0 + j);
            double g[16];
#pragma unroll
            for (int t = 0; t < 16; t++) {
                int i = a + t;
                i = i >= nf ? i - nf : i;
                g[t] = t < w ? __ldg(grid + i) : 0.0;
            }
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t < 16; t++)
                if (t < w) acc = fma(g[t], ks[threadIdx.x * w + t], acc);
            u[j] = acc;
        }
    }
}

// mixed interpolation (A6) by units: the block converts the unit's grid span to FP32 in shared
// memory once, then each thread sums its point's w taps in FP32 (rounding errors of the order of
// the kernel's fit, below the requested tolerance)
template <int D>
__global__ void __launch_bounds__(kUnitPoints) k_nu_interp_mixed(const NuUnit* __restrict__ units,
                                                                 const double* __restrict__ grid,
                                                                 double* __restrict__ u,
                                                                 const int32_t* __restrict__ first,
                                                                 const float* __restrict__ soff, const NuPoly P,
                                                                 int w, int nf) {
    __shared__ float gs[kUnitCells + 16];
    const NuUnit un = units[blockIdx.x];
    for (int l = threadIdx.x; l < un.span; l += kUnitPoints) gs[l] = nu_f64_to_f32(__ldg(grid + (un.ca + l) % nf));
    __syncthreads();
    const int p = threadIdx.x;
    if (p < un.np) {
        const int64_t j = (int64_t)un.pa + p;
        const int a = __ldg(first + j) - un.ca;
        const float y = __fmaf_rn(2.f, __ldcs(soff + j), -1.f);
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < 16; t++)
            if (t < w) acc = __fmaf_rn(nu_psi<D>(P.c[t], y), gs[a + t], acc);
        __stcs(u + j, nu_f32_to_f64(acc));
    }
}

// polynomial degrees the mixed kernels are built for
template <typename F>
bool nu_with_degree(int D, F&& f) {
    switch (D) {
        case 6: f(std::integral_constant<int, 6>{}); return true;
        case 8: f(std::integral_constant<int, 8>{}); return true;
        case 10: f(std::integral_constant<int, 10>{}); return true;
        case 12: f(std::integral_constant<int, 12>{}); return true;
        case 14: f(std::integral_constant<int, 14>{}); return true;
        case 16: f(std::integral_constant<int, 16>{}); return true;
        default: return false;
    }
}

int ilog2n(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// least-squares monomial fit of degree D in y in [-1, 1] to f at n Chebyshev points (normal
// equations in long double; D <= 16 and smooth f)
std::vector<double> fit_poly(const std::vector<double>& ys, const std::vector<double>& fs, int D) {
    const int n = (int)ys.size(), m = D + 1;
    std::vector<long double> A((size_t)m * m, 0.0L), b(m, 0.0L);
    for (int i = 0; i < n; i++) {
        long double p[kMaxDegree + 1];
        p[0] = 1.0L;
        for (int d = 1; d < m; d++) p[d] = p[d - 1] * (long double)ys[i];
        for (int r = 0; r < m; r++) {
            b[r] += p[r] * (long double)fs[i];
            for (int q = 0; q < m; q++) A[(size_t)r * m + q] += p[r] * p[q];
        }
    }
    // Gaussian elimination with partial pivoting
    for (int col = 0; col < m; col++) {
        int piv = col;
        for (int r = col + 1; r < m; r++)
            if (std::fabs((double)A[(size_t)r * m + col]) > std::fabs((double)A[(size_t)piv * m + col])) piv = r;
        if (piv != col) {
            for (int q = 0; q < m; q++) std::swap(A[(size_t)col * m + q], A[(size_t)piv * m + q]);
            std::swap(b[col], b[piv]);
        }
        for (int r = col + 1; r < m; r++) {
            long double f = A[(size_t)r * m + col] / A[(size_t)col * m + col];
            for (int q = col; q < m; q++) A[(size_t)r * m + q] -= f * A[(size_t)col * m + q];
            b[r] -= f * b[col];
        }
    }
    std::vector<double> c(m, 0.0);
    for (int r = m - 1; r >= 0; r--) {
        long double s = b[r];
        for (int q = r + 1; q < m; q++) s -= A[(size_t)r * m + q] * (long double)c[q];
        c[r] = (double)(s / A[(size_t)r * m + r]);
    }
    return c;
}

}  // namespace

struct wave1d_nufft_s {
    int device = 0;
    int precision = 0;
    int64_t M = 0;
    Params P{};
    int D = 0;                       // polynomial degree (mixed)
    double kernel_err = 0.0;         // max |polynomial (FP32 Horner) - kernel| over the taps (mixed)
    cudaStream_t stream = nullptr;
    std::vector<int64_t> perm;       // internal point i -> caller index
    std::vector<void*> allocs;
    // points (internal order): first cell, offset in it (mixed), kernel weights (FP64)
    int32_t* first = nullptr;
    float* soff = nullptr;
    NuPoly poly{};                   // tap polynomials (mixed), passed to the kernels by value
    double* ker = nullptr;
    // spreading units and the cells' partials
    NuUnit* units = nullptr;
    int64_t nunits = 0;
    double* partial = nullptr;
    int32_t *cptr = nullptr, *cent = nullptr;
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

extern "C" {

int wave1d_nufft_plan(const double* x, int64_t M, int K, double tol, int precision, void* stream,
                      wave1d_nufft_t* out) {
    if (!out) return nfail(WAVE1D_EINVAL, "out is NULL");
    *out = nullptr;
    if (!x || M < 1 || M > INT32_MAX / 32 || K < 1 || !(tol > 0.0 && tol < 0.1) || (precision != 0 && precision != 1))
        return nfail(WAVE1D_EINVAL, "need x, 1 <= M < 2^26, K >= 1, 0 < tol < 0.1, precision 0 or 1");
    wave1d_nufft_t h = new (std::nothrow) wave1d_nufft_s();
    if (!h) return nfail(WAVE1D_ENOMEM, "host allocation");
    auto cleanup = [&](int code) {
        wave1d_nufft_destroy(h);
        return code;
    };
    h->precision = precision;
    h->M = M;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) return cleanup(nfail(WAVE1D_ECUDA, "no CUDA device"));
    Params& P = h->P;
    nufft_grid(P, K, tol, 0);
    if (P.L2 > 1024) return cleanup(nfail(WAVE1D_EUNSUPPORTED, "fine grid too large for this build (nf > 2^21)"));
    const int w = P.nufft_w, nf = P.nf;
    // positions wrapped into [-pi, pi), kernel weights, internal order by first cell
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
    std::stable_sort(h->perm.begin(), h->perm.end(), [&](int64_t a, int64_t b) {
        return i0c[a] != i0c[b] ? i0c[a] < i0c[b] : xw[a] < xw[b];
    });
    std::vector<int32_t> i0(M);
    std::vector<double> xs(M);
    for (int64_t i = 0; i < M; i++) {
        i0[i] = i0c[h->perm[i]];
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
            double u = (xs[i] + kPiN) / P.h_f;
            double fst = std::ceil(u - 0.5 * w);
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
        // degrees 6, 8, ..., 16 (the ones the kernels are built for): the first within 2e-7
        int D = 6;
        double err = 1.0;
        for (;; D += 2) {
            err = 0.0;
            for (int t = 0; t < w; t++) {
                std::vector<double> fs(ns);
                for (int i = 0; i < ns; i++) fs[i] = kernel(ys[i], t);
                std::vector<double> c = fit_poly(ys, fs, D);
                for (int d = 0; d <= kMaxDegree; d++) h->poly.c[t][d] = d <= D ? (float)c[d] : 0.f;
                for (int i = 0; i <= 400; i++) {          // FP32 Horner, as on the device
                    float y = (float)(-1.0 + 2.0 * i / 400.0);
                    float r = h->poly.c[t][D];
                    for (int d = D - 1; d >= 0; d--) r = std::fma(r, y, h->poly.c[t][d]);
                    err = std::max(err, std::fabs((double)r - kernel((double)y, t)));
                }
            }
            if (err < 2e-7 || D == kMaxDegree) break;
        }
        h->D = D;
        h->kernel_err = err;
        if ((rc = nu_upload(h, soff, &h->soff))) return cleanup(rc);
    }
    // spreading units: runs of at most kUnitPoints points whose first cells span < kUnitCells
    // cells; each reaches its cells plus w - 1 (wrapped into the grid by the combine pass)
    {
        std::vector<NuUnit> units;
        int64_t poff = 0;
        for (int64_t a = 0; a < M;) {
            int64_t b = a + 1;
            while (b < M && b - a < kUnitPoints && i0[b] - i0[a] < kUnitCells) b++;
            NuUnit u{};
            u.pa = (int32_t)a;
            u.np = (int32_t)(b - a);
            u.ca = i0[a];
            u.span = i0[b - 1] - i0[a] + w;
            u.poff = (int32_t)poff;
            poff += u.span;
            units.push_back(u);
            a = b;
        }
        std::vector<int32_t> cptr(nf + 1, 0);
        for (const NuUnit& u : units)
            for (int l = 0; l < u.span; l++) cptr[(u.ca + l) % nf + 1]++;
        for (int r = 0; r < nf; r++) cptr[r + 1] += cptr[r];
        std::vector<int32_t> cent(cptr[nf]), fill(cptr.begin(), cptr.end() - 1);
        for (const NuUnit& u : units)
            for (int l = 0; l < u.span; l++) cent[fill[(u.ca + l) % nf]++] = u.poff + l;
        h->nunits = (int64_t)units.size();
        if ((rc = nu_upload(h, units, &h->units)) || (rc = nu_upload(h, cptr, &h->cptr)) ||
            (rc = nu_upload(h, cent, &h->cent)) || (rc = nu_alloc(h, (size_t)poff, &h->partial)) ||
            (rc = nu_upload(h, i0, &h->first)))
            return cleanup(rc);
    }
    std::vector<double> d1, d2, mf, tw((size_t)P.L * 2);
    nufft_factors(P, d1, d2, mf);
    for (int j = 0; j < P.L; j++) {
        double a = 2.0 * kPiN * (double)j / (double)P.L;
        tw[2 * j] = std::cos(a);
        tw[2 * j + 1] = std::sin(a);
    }
    if ((rc = nu_upload(h, mf, &h->modefac)) || (rc = nu_upload(h, tw, &h->twiddle)) ||
        (rc = nu_alloc(h, (size_t)nf, &h->grid)) || (rc = nu_alloc(h, (size_t)nf, &h->work)) ||
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
    const int nf = h->P.nf, w = h->P.nufft_w;
    const unsigned nu = (unsigned)h->nunits, nc = (unsigned)((nf + 255) / 256);
    if (h->precision == 0) {
        k_nu_spread64<<<nu, kUnitPoints, 0, h->stream>>>(h->units, c, h->first, h->ker, w, h->partial);
        k_nu_combine64<<<nc, 256, 0, h->stream>>>(h->partial, h->cptr, h->cent, grid, nf);
    } else {
        float2* part = reinterpret_cast<float2*>(h->partial);
        nu_with_degree(h->D, [&](auto dc) {
            k_nu_spread_mixed<decltype(dc)::value><<<nu, kUnitPoints, 0, h->stream>>>(h->units, c, h->first, h->soff,
                                                                                    h->poly, w, part);
        });
        k_nu_combine32<<<nc, 256, 0, h->stream>>>(part, h->cptr, h->cent, grid, nf);
    }
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "spread launch failed");
}

int wave1d_nufft_interp(wave1d_nufft_t h, const double* grid, double* u) {
    if (!h || !grid || !u) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    const unsigned nb = (unsigned)std::min<int64_t>((h->M + 255) / 256, 1 << 20);
    if (h->precision == 0)
        k_nu_interp64<<<nb, 256, 0, h->stream>>>(grid, u, h->first, h->ker, h->M, h->P.nufft_w, h->P.nf);
    else
        nu_with_degree(h->D, [&](auto dc) {
            k_nu_interp_mixed<decltype(dc)::value><<<(unsigned)h->nunits, kUnitPoints, 0, h->stream>>>(
                h->units, grid, u, h->first, h->soff, h->poly, h->P.nufft_w, h->P.nf);
        });
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "interp launch failed");
}

int wave1d_nufft_type1(wave1d_nufft_t h, const double* c, double* S) {
    if (!h || !c || !S) return nfail(WAVE1D_EINVAL, "bad arguments");
    int rc = wave1d_nufft_spread(h, c, h->grid);
    if (rc) return rc;
    const Params& P = h->P;
    const int t1 = std::max(32, std::min(P.L1 / 2, 512)), t2 = std::max(32, std::min(P.L2 / 2, 512));
    k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), h->stream>>>((const double2*)h->grid, (double2*)h->work,
                                                              (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                              ilog2n(P.L1), +1);
    k_fft_rows<<<P.L1, t2, fft_smem_bytes(P.L2), h->stream>>>((const double2*)h->work, (double2*)h->spec,
                                                              (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                              ilog2n(P.L2), +1);
    k_nu_post1<<<(P.K + 1 + 127) / 128, 128, 0, h->stream>>>((const double2*)h->spec, S, h->modefac, P.K, P.L);
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : nfail(WAVE1D_ECUDA, "type-1 launch failed");
}

int wave1d_nufft_type2(wave1d_nufft_t h, const double* alpha, double* u) {
    if (!h || !alpha || !u) return nfail(WAVE1D_EINVAL, "bad arguments");
    if (cudaSetDevice(h->device) != cudaSuccess) return nfail(WAVE1D_ECUDA, "cudaSetDevice");
    const Params& P = h->P;
    k_nu_pre2<<<(P.L + 255) / 256, 256, 0, h->stream>>>(alpha, (double2*)h->spec2, h->modefac, P.K, P.L);
    const int t1 = std::max(32, std::min(P.L1 / 2, 512)), t2 = std::max(32, std::min(P.L2 / 2, 512));
    k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), h->stream>>>((const double2*)h->spec2, (double2*)h->work,
                                                              (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                              ilog2n(P.L1), -1);
    k_fft_rows<<<P.L1, t2, fft_smem_bytes(P.L2), h->stream>>>((const double2*)h->work, (double2*)h->grid,
                                                              (const double2*)h->twiddle, P.L, P.L1, P.L2,
                                                              ilog2n(P.L2), -1);
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

const char* wave1d_nufft_strerror(void) { return g_nu_error.c_str(); }

}  // extern "C"
