// Per-stage kernels of the WFP march, one launch per stage.  Ordinary steps normally run as the
// one-launch step kernel (step.cu); these kernels run projection steps, profiled steps and plans
// that ask for per-stage launches.  One time step n -> n+1:
//   k_local_items local explicit sum over the last delta of history (Sec. 4.1, m >= 1)
//   history pipeline (history.cu): spreading + forward FFT columns, forward FFT rows + mode
//                 update (Sec. 3) + inverse FFT rows, inverse FFT columns
//   [k_rbc_grid, k_rbc_update, k_fft_cols, k_fft_rows]  on projection steps (Sec. 4.4) the
//                 projection and the inverse FFT of the natural-order type-2 spectrum
//   k_interp      u_H at springs and receivers (eq. historySol1 via NUFFT)
//   k_solve       right-hand side and block solve of eq. linearSystem; its last block reads out
//                 the receivers (u = u_L + u_H) and advances the step counter
// Kernels read the step index n from device memory so that captured graphs can be replayed.
//
// GB300 runs FP64 at about 2 FMA per clock per SM and FP32 at 128, so the one phase with a
// per-pair inner loop (the local sum) does its products and sums in compensated FP32 pairs
// (hi + lo, about 48 significant bits), which keeps it bound by HBM rather than by the FP64 pipe.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {

__global__ void __launch_bounds__(256, 4) k_local_items(DevPlan P) { local_items_loop(P, load_step(P)); }

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


__global__ void k_interp(DevPlan P) {
    const int64_t n = load_step(P), nchunks = (P.M + P.R + kInterpPoints - 1) / kInterpPoints;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) interp_chunk(P, n, c, nullptr);
}

__global__ void __launch_bounds__(256) k_solve(DevPlan P) {
    __shared__ double srhs[8][kSolveStage];
    __shared__ bool last;
    int64_t n = load_step(P);
    int wid = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.item_ctr = 0ull;   // the step's local sums are done
    solve_tasks(P, n, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                 ((int64_t)gridDim.x * blockDim.x) >> 5, srhs[wid]);
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
