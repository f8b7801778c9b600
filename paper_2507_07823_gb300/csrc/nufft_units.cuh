// One block's unit of the FP64 spreading and interpolation passes of the history part (Sec. 3.1:
// eq. densco spreads the densities onto the fine grid, eq. historySol1's interpolation reads it
// back at the points), shared by the standalone NUFFT kernels (nufft.cu) and the batched one-launch
// step (batch_step.cu).  A call is one block's work on one unit; the block's threads all call it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "nufft_host.h"
#include "../../include/wave1d.h"

namespace wave1d {

constexpr int kUnitThreads = 256;   // threads of a spreading block
constexpr int kRangeCells64 = 128;  // cells of an FP64 range (its w tap sums per cell live in shared memory)
constexpr int kInterpTile = 256;    // points of an FP64 interpolation tile

// shared memory of the units: the run table and the w tap sums of every cell of a range; the
// staged weights of a tile of points (up to 16 taps)
constexpr int kSpread64Runs = kRangeCells64 + 16 + 1;
template <int W>
constexpr size_t spread64_smem() {
    return (size_t)(kRangeCells64 + 16) * W * sizeof(double) + (size_t)(kSpread64Runs + 1) * sizeof(int);
}
constexpr size_t kInterp64Smem = (size_t)kInterpTile * 16 * sizeof(double);

// FP64 spreading of range u on the cell ranges of the plan: each cell's lanes accumulate the w tap
// sums S_t(f) = sum_{q: i0_q = f} ker_q[t] c_q (one FMA per point and tap, weights and densities
// read four points at a time), a fixed shuffle tree closes each group, and grid real c0 + l =
// sum_t S_t(c0 + l - t).  seg: (kRangeCells64 + 16) x W doubles; rp: kSpread64Runs ints.  No block
// depends on another; the block synchronises on entry, so consecutive units may reuse the buffers.
template <int W>
__device__ __forceinline__ void spread64_unit(const NuRange& u, const int32_t* __restrict__ runs,
                                              const double* __restrict__ c, const double* __restrict__ ker,
                                              double* __restrict__ grid, double (*seg)[W], int* rp) {
    __syncthreads();
    const int nr = u.nc + W - 1, np = u.na + u.nb;
    if (np == 0) {
        for (int l = threadIdx.x; l < u.nc; l += blockDim.x) grid[u.c0 + l] = 0.0;
        return;
    }
    if ((int)threadIdx.x <= nr) rp[threadIdx.x] = __ldg(runs + u.roff + threadIdx.x);
    __syncthreads();
    const int G = 1 << u.lg, f = (int)threadIdx.x >> u.lg, gl = (int)threadIdx.x & (G - 1);
    double acc[W];
#pragma unroll
    for (int t = 0; t < W; t++) acc[t] = 0.0;
    if (f < nr) {
        const int q1 = rp[f + 1];
        constexpr int B = 4;
        for (int q = rp[f] + gl; q < q1; q += B * G) {
            double cb[B], kb[B][W];
#pragma unroll
            for (int i = 0; i < B; i++) {
                const int qi = q + i * G < q1 ? q + i * G : q;
                const int64_t j = qi < u.na ? u.a0 + qi : u.b0 + (qi - u.na);
                cb[i] = q + i * G < q1 ? __ldcs(c + j) : 0.0;
#pragma unroll
                for (int t = 0; t < W; t++) kb[i][t] = __ldcs(ker + j * W + t);
            }
#pragma unroll
            for (int i = 0; i < B; i++)
#pragma unroll
                for (int t = 0; t < W; t++) acc[t] = fma(kb[i][t], cb[i], acc[t]);
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
        for (int t = 0; t < W; t++) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    }
    if (gl == 0 && f < nr) {
#pragma unroll
        for (int t = 0; t < W; t++) seg[f][t] = acc[t];
    }
    __syncthreads();
    if ((int)threadIdx.x < u.nc) {
        const int l = threadIdx.x;
        double a = 0.0;
        if (rp[l + W] != rp[l]) {                     // else none of the w cells feeding it holds a point
#pragma unroll
            for (int t = 0; t < W; t++) a += seg[l + W - 1 - t][t];
        }
        grid[u.c0 + l] = a;
    }
}

// FP64 interpolation of tile t (points t kInterpTile ..): u_j = sum_u G[(i0_j + u) mod nf] ker[j][u]
// (i0_j: instance x nf + cell).  The tile's weights (one contiguous run of np w doubles) are staged
// through ks (kInterpTile x 16 doubles) with coalesced streaming loads, and all w grid loads of a
// point are issued before any is used.  The block synchronises on entry and after staging.
__device__ __forceinline__ void interp64_unit(int64_t t, const double* __restrict__ grid, double* __restrict__ u,
                                              const int32_t* __restrict__ i0, const double* __restrict__ ker,
                                              int64_t M, int w, int nf, double* ks) {
    const int64_t base = t * kInterpTile;
    const int np = (int)(M - base < kInterpTile ? M - base : kInterpTile);
    __syncthreads();
    const double* kr = ker + base * w;
    for (int e = threadIdx.x; e < np * w; e += blockDim.x) ks[e] = __ldcs(kr + e);
    __syncthreads();
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int64_t j = base + p;
        const int a = __ldg(i0 + j), gb = a & ~(nf - 1);   // instance x nf + cell
        double g[16];
#pragma unroll
        for (int q = 0; q < 16; q++) g[q] = q < w ? __ldg(grid + (gb | ((a + q) & (nf - 1)))) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 16; q++)
            if (q < w) acc = fma(g[q], ks[p * w + q], acc);
        u[j] = acc;
    }
}

// The device arrays of an FP64 NUFFT plan that the unit bodies read (for kernels outside nufft.cu)
struct NuDev64 {
    const NuRange* ranges;
    const int32_t* runs;
    int64_t nunits;          // spreading ranges
    const double* ker;       // M x w kernel weights
    const int32_t* i0;       // first cell of each point (instance x nf + cell)
    int64_t M;
    int w, nf;
};
// WAVE1D_EINVAL for a plan that is not FP64 (defined in nufft.cu)
int nufft_dev64(wave1d_nufft_t h, NuDev64& out);

}  // namespace wave1d
