// Kernels of the reverse-time (adjoint) march: the transposed pieces of one step, each a thin
// launch around a body of adjoint.cuh (the derivation is at the top of that file).  The type-1
// and type-2 transforms of the reverse step run through a standalone NUFFT plan on the springs.
//
// Adjoint state (internal spring order):
//   sb   ring of m_max + 1 slots x M: sigmabar^q in slot q mod (m_max + 1)
//   Sb   ring of W slots x (K + 1) complex: Sbar^q in slot q mod W
//   ab, apb  alphabar, alpha'bar (K + 1 complex)
// Contributions to sb from different targets or receivers meet at the same source, so they are
// added with atomics (the gradient is then reproducible to rounding, not bit for bit).
#include <cuda_runtime.h>

#include <cstdint>

#include "adjoint.cuh"
#include "internal.h"

namespace wave1d {

// receivers: warps [0, r_nitems) take one receiver item each (m >= 1 slices), warps
// [r_nitems, r_nitems + R) the m = 0 terms of one receiver (sources closer than dt).  The row of
// an item is found in r_item_ptr (R + 1 offsets) by bisection.
__global__ void k_adj_receivers(DevPlan P, int64_t n, const double* __restrict__ ubar, double* sb) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t q = n + 1;
    if (gw < P.r_nitems) {
        int64_t lo = 0, hi = P.R;                   // r_item_ptr[lo] <= gw < r_item_ptr[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (P.r_item_ptr[mid] <= gw) lo = mid;
            else hi = mid;
        }
        const double coef = 0.5 * ubar[lo];
        if (coef == 0.0) return;
        const int src = P.r_src[gw * 32 + lane];
        adj::item_lane_T(P.r_w, P.r_wbase[gw], P.r_s0[gw], P.r_len[gw], lane, src, P.r_mfirst, coef, q,
                         P.ring, [&](int s, int j, double v) { atomicAdd(sb + (int64_t)s * P.M + j, v); });
    } else if (gw < P.r_nitems + P.R) {
        const int64_t r = gw - P.r_nitems;
        const double coef = 0.5 * ubar[r];
        double* s1 = sb + (int64_t)adj::slot(q, P.ring) * P.M;
        for (int e = lane; e < P.r0_stride; e += 32) {
            const double w = P.r0p_w[r * P.r0_stride + e];
            if (w != 0.0) atomicAdd(s1 + P.r0p_src[r * P.r0_stride + e], w * coef);
        }
    }
}

// sigmabar^{n+1} is complete: move it out of its ring slot (which becomes sigma^{n-m_max}'s)
__global__ void k_adj_take(int64_t M, double* __restrict__ slot_vals, double* __restrict__ out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        out[j] = slot_vals[j];
        slot_vals[j] = 0.0;
    }
}

// transposed block solve, one thread per member position e of blk_members (blk_of[e] = its
// block), then the step's gradient term and the adjoints of the local sum and of u_H:
//   grad_j += rhsbar_j sigma_j^{n+1} / beta_j,  cbar_j = -beta_j rhsbar_j / 2,  u_Hbar_j = -beta_j rhsbar_j
__global__ void k_adj_solve(DevPlan P, const int32_t* __restrict__ blk_of, const double* __restrict__ sigbar,
                            const double* __restrict__ sigma_next, double* grad, double* cbar, double* uHbar) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.M; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = blk_of[e];
        const int64_t m0 = P.blk_ptr[b];
        const int s = (int)(P.blk_ptr[b + 1] - m0);
        const double rb = adj::solve_T(P.inv + P.blk_inv_off[b], P.blk_members, m0, s, (int)(e - m0), sigbar);
        const int j = P.blk_members[e];
        const double bj = P.beta[j];
        grad[j] += rb * sigma_next[P.perm[j]] / bj;
        cbar[j] = -0.5 * bj * rb;
        uHbar[j] = -bj * rb;
    }
}

// transposed local sum of the springs: one warp per item of the step layout
__global__ void k_adj_local(DevPlan P, int64_t n, const double* __restrict__ cbar, double* sb) {
    const int lane = threadIdx.x & 31;
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (o >= P.l_nitems) return;
    const double coef = cbar[P.l_row[o]];
    if (coef == 0.0) return;
    const int src = P.l_src[o * 32 + lane];
    adj::item_lane_T(P.l_w, P.l_wbase[o], P.l_s0[o], P.l_len[o], lane, src, P.l_mfirst, coef, n + 1, P.ring,
                     [&](int s, int j, double v) { atomicAdd(sb + (int64_t)s * P.M + j, v); });
}

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

}  // namespace wave1d
