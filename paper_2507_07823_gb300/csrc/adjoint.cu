// Kernels of the reverse-time (adjoint) march: the transposed pieces of one step, each a thin
// launch around a body of adjoint.cuh (the derivation is at the top of that file).  The type-1
// and type-2 transforms of the reverse step run through a standalone NUFFT plan on the springs.
//
// Adjoint state (internal spring order):
//   sb   ring of m_max + 1 slots x M: sigmabar^q in slot q mod (m_max + 1)
//   Sb   ring of W slots x (K + 1) complex: Sbar^q in slot q mod W
//   ab, apb  alphabar, alpha'bar (K + 1 complex)
// Every launch has one writer per output element and sums in a fixed order: no atomics, and the
// gradient is the same bit for bit from run to run.
#include <cuda_runtime.h>

#include <cstdint>

#include "adjoint.cuh"
#include "internal.h"

namespace wave1d {

// receivers' transposed readout, one thread per source over the receiver weights regrouped by
// source (m >= 0: the m = 0 terms of sources closer than dt included)
__global__ void k_adj_receivers(int64_t M, int ring, int64_t n, const int64_t* __restrict__ ptr,
                                const int32_t* __restrict__ rcv, const int32_t* __restrict__ mrange,
                                const int64_t* __restrict__ woff, const double* __restrict__ w,
                                const double* __restrict__ ubar, double* sb) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < M; l += (int64_t)gridDim.x * blockDim.x)
        adj::receivers_T_source(l, ptr, rcv, mrange, woff, w, ubar, n + 1, ring,
                                [&](int s, double v) { sb[(int64_t)s * M + l] += v; });
}

// sigmabar^{n+1} is complete: move it out of its ring slot (which becomes sigma^{n-m_max}'s)
__global__ void k_adj_take(int64_t M, double* __restrict__ slot_vals, double* __restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        out[j] = slot_vals[j];
        slot_vals[j] = 0.0;
    }
}

// transposed block solve, one thread per member position e of blk_members (blk_of[e] = its
// block), then the step's gradient terms and the adjoints of the local sum and of u_H:
//   grad_j += rhsbar_j (sigma_j^{n+1} + g_j^{n+1}) / beta_j   (g: a forcing that does not scale
//             with beta; for the incident wave g = beta f is part of rhs and the term is
//             rhsbar_j sigma_j^{n+1} / beta_j),
//   gbar_j^{n+1} = -rhsbar_j,  cbar_j = -beta_j rhsbar_j / 2,  u_Hbar_j = -beta_j rhsbar_j.
// sigma_next, g_next and gbar_next are rows in caller order; g_next, grad and gbar_next may be null.
__global__ void k_adj_solve(DevPlan P, const int32_t* __restrict__ blk_of, const double* __restrict__ sigbar,
                            const double* __restrict__ sigma_next, const double* __restrict__ g_next, double* grad,
                            double* __restrict__ gbar_next, double* cbar, double* uHbar) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.M; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = blk_of[e];
        const int64_t m0 = P.blk_ptr[b];
        const int s = (int)(P.blk_ptr[b + 1] - m0);
        const double rb = adj::solve_T(P.inv + P.blk_inv_off[b], P.blk_members, m0, s, (int)(e - m0), sigbar);
        const int j = P.blk_members[e];
        const int jc = P.perm[j];
        const double bj = P.beta[j];
        if (grad) grad[j] += rb * (g_next ? sigma_next[jc] + g_next[jc] : sigma_next[jc]) / bj;
        if (gbar_next) gbar_next[jc] = -rb;
        cbar[j] = -0.5 * bj * rb;
        uHbar[j] = -bj * rb;
    }
}

// transposed local sum of the springs, one warp per row l (the row's items read in the transposed
// direction, Q_m being symmetric in the pair), in the compensated FP32 arithmetic of the forward
// local sum: each lane accumulates its slices into the warp's shared pairs acc[m][lane] (row
// stride kAdjAccStride), then lane i adds m = i, i + 32, ... over the 32 lanes in lane order (in
// FP64) and adds the result to sigmabar^{n+1-m}[l].  Dynamic shared memory: warps per block x
// (m_max + 1) x kAdjAccStride float pairs.
constexpr int kAdjAccStride = 33;

__global__ void k_adj_local(DevPlan P, int64_t n, const double* __restrict__ cbar, double* sb) {
    extern __shared__ float2 adj_acc[];
    const int lane = threadIdx.x & 31;
    const int nm = P.m_max + 1;
    float2* acc = adj_acc + (int64_t)(threadIdx.x >> 5) * nm * kAdjAccStride;
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= P.M) return;                                  // the whole warp: l is the warp's row
    for (int m = 0; m < nm; m++) acc[m * kAdjAccStride + lane] = make_float2(0.f, 0.f);
    for (int64_t it = P.l_item_ptr[l]; it < P.l_item_ptr[l + 1]; it++) {
        float ch, cl;
        adj::split_pair(cbar[P.l_src[it * 32 + lane]], ch, cl);
        adj::item_lane_gather(P.l_w, P.l_wbase[it], P.l_s0[it], P.l_len[it], lane, P.l_mfirst, ch, cl,
                              [&](int m) { return (float*)(acc + m * kAdjAccStride + lane); });
    }
    __syncwarp();
    for (int m = lane; m < nm; m += 32) {
        double s = 0.0;
        for (int i = 0; i < 32; i++) {
            const float2 a = acc[m * kAdjAccStride + i];
            s += (double)a.x + (double)a.y;
        }
        if (s != 0.0) sb[(int64_t)adj::slot(n + 1 - m, P.ring) * P.M + l] += s;
    }
}

size_t adj_local_smem(int m_max, int warps) { return (size_t)warps * (m_max + 1) * kAdjAccStride * sizeof(float2); }

// out[i] = in[perm[i]] (spring order -> NUFFT point order)
__global__ void k_adj_gather(int64_t M, const int64_t* __restrict__ perm, const double* __restrict__ in,
                             double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

// acc[perm[i]] += in[i] (NUFFT point order -> spring order; perm is a permutation)
__global__ void k_adj_scatter_add(int64_t M, const int64_t* __restrict__ perm, const double* __restrict__ in,
                                  double* __restrict__ acc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        acc[perm[i]] += in[i];
}

__global__ void k_adj_modes_in(int K, const double* __restrict__ S1, const double* __restrict__ xr,
                               const double* __restrict__ ubar, int64_t R, double* ab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) adj::modes_in(k, S1, xr, ubar, R, ab);
}

__global__ void k_adj_rbc_grid(int K, int npts, const int32_t* __restrict__ idx, const double* __restrict__ tw2K,
                               const double* __restrict__ phi, const double* __restrict__ dphi,
                               const double* __restrict__ ab, const double* __restrict__ apb,
                               double* __restrict__ uvbar) {
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    if (pt < npts) adj::rbc_grid_T(idx[pt], K, tw2K, ab, apb, phi[pt], dphi[pt], uvbar + 2 * pt, uvbar + 2 * pt + 1);
}

__global__ void k_adj_rbc_update(int K, int npts, const int32_t* __restrict__ idx, const double* __restrict__ tw2K,
                                 const double* __restrict__ uvbar, double* ab, double* apb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) adj::rbc_update_T(k, K, npts, idx, tw2K, uvbar, ab, apb);
}

__global__ void k_adj_modes(int K, int W, int64_t n, const double* __restrict__ rot, const double* __restrict__ pq,
                            double* ab, double* apb, double* Sb, double* __restrict__ a2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) adj::modes_T(k, K + 1, W, n, rot, pq, ab, apb, Sb, a2);
}

// Checkpoint restore (wave1d_adjoint_checkpointed): the float-pair copy of the density ring
// (both halves of its doubled ring) from the FP64 ring, the same split store_sigma makes, so a
// march resumed from a checkpoint of the FP64 ring alone repeats the original bit for bit
__global__ void k_ck_sig2(int64_t n, const double* __restrict__ sig, float2* __restrict__ sig2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = sig[i];
        const float hi = (float)v;
        const float2 pr = make_float2(hi, (float)(v - (double)hi));
        sig2[i] = pr;
        sig2[i + n] = pr;
    }
}

// the device step counter of a restored march
__global__ void k_ck_step(int64_t* step, int64_t n) {
    step[0] = n;
    step[1] = 0;
}

}  // namespace wave1d
