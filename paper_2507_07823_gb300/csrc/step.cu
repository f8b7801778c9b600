// One ordinary time step n -> n+1 of the WFP march as a single cooperative launch.
//
// The step has two independent halves that both start from sigma^{<= n}: the local explicit sum
// (Sec. 4.1), which streams the stored weights and is bound by HBM, and the history pipeline
// (Sec. 3: type-1 NUFFT, mode update, type-2 NUFFT, interpolation), a chain of short latency-bound
// passes.  As separate launches they run back to back, each short pass paying a launch and a
// ramp.  Here both run at once:
//
//   blocks [0, hist_blocks)  the history pipeline, its columns, row pairs, inverse columns and
//                            point chunks handed out by counters, each phase waiting for the one
//                            before, then the FIR tail of the next step; then local items
//   other blocks             the forcing of the step (chunks of springs), then local sum items
//                            (atomic counter); then whatever history work is left
//   all blocks               grid barrier; block solve of eq. linearSystem; the block that
//                            finishes last resets the counters, reads out the receivers and
//                            advances the step counter
//
// The history blocks are consecutive block indices, which the hardware spreads over different
// SMs: their FP64 work (GB300 issues one FP64 warp instruction per 64 cycles per SM partition)
// then uses many SMs' FP64 units, which the local sum (FP32 and loads) leaves idle.  Work is taken,
// not assigned, so the step completes wherever the blocks run.  Every block is resident (the launch
// is cooperative) and every wait is bounded: a wait that runs out latches WAVE1D_ETIMEOUT in the
// status word and the block returns; the other blocks then give up at their next wait.
// Projection steps (Sec. 4.4) use the per-stage kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {

// polls of a counter before a wait gives up (each poll sleeps about 0.1-1 us)
constexpr unsigned kSpinLimit = 1u << 22;

// counters in P.bar (all zero between steps)
enum : int {
    kColTake = 0, kColDone, kRowTake, kRowDone, kIcolTake, kIcolDone, kIntTake, kTailTake,
    kForceTake, kForceDone, kGrid, kNumCounters
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0 waits until *ctr >= target; false if the wait ran out (or another block's did).  The
// block synchronises before and after.
__device__ __forceinline__ bool wait_for(const DevPlan& P, const unsigned* ctr, unsigned target) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        unsigned polls = 0;
        while (ld_acquire(ctr) < target) {
            if (++polls > kSpinLimit) {
                atomicCAS(P.status, 0, (int)WAVE1D_ETIMEOUT);
                good = 0;
                break;
            }
            if ((polls & 255u) == 0 && *(volatile int*)P.status == (int)WAVE1D_ETIMEOUT) {
                good = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// the block takes the next unit of a phase (broadcast to all its threads)
__device__ __forceinline__ unsigned take(unsigned* ctr) {
    __shared__ unsigned t;
    __syncthreads();
    if (threadIdx.x == 0) t = atomicAdd(ctr, 1u);
    __syncthreads();
    return t;
}

// the block's writes of a finished unit become visible before the unit is counted
__device__ __forceinline__ void finish(unsigned* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

// The small working set of the later phases (FIR taps and history ring, per-mode factors,
// interpolation kernels, block inverses: a few MB) is pulled into L2 after the column pass, so the
// latency-bound phases that follow find it there.
__device__ __forceinline__ void prefetch_step_state(const DevPlan& P, int64_t tid, int64_t nt) {
    const size_t K1 = (size_t)P.K + 1, M = (size_t)P.M, R = (size_t)P.R, w = (size_t)P.w;
    prefetch_l2(P.twiddle, (size_t)P.L * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.Sring, (size_t)P.W * K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.pq, (size_t)P.W * K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.modefac, K1 * 8 * sizeof(double), tid, nt);
    prefetch_l2(P.rot, K1 * 3 * sizeof(double), tid, nt);
    prefetch_l2(P.alpha, K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.alpha_p, K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.sp_i0, M * sizeof(int32_t), tid, nt);
    prefetch_l2(P.sp_ker, M * w * sizeof(double), tid, nt);
    prefetch_l2(P.x, M * sizeof(double), tid, nt);
    prefetch_l2(P.beta, M * sizeof(double), tid, nt);
    if (R) {
        prefetch_l2(P.rc_i0, R * sizeof(int32_t), tid, nt);
        prefetch_l2(P.rc_ker, R * w * sizeof(double), tid, nt);
    }
    prefetch_l2(P.blk_ptr, ((size_t)P.nblocks + 1) * sizeof(int64_t), tid, nt);
    prefetch_l2(P.blk_inv_off, ((size_t)P.nblocks + 1) * sizeof(int64_t), tid, nt);
    prefetch_l2(P.blk_members, M * sizeof(int32_t), tid, nt);
    prefetch_l2(P.inv, (size_t)P.inv_len * sizeof(double), tid, nt);
    prefetch_l2(P.l_item_ptr, (M + 1) * sizeof(int64_t), tid, nt);
}

// forcing g_j(t_{n+1}) of the step's springs, computed ahead in chunks of blockDim springs (its
// FP64 exponentials stay off the history chain)
__device__ __forceinline__ void forcing_units(const DevPlan& P, int64_t n) {
    unsigned* c = P.bar;
    const unsigned nforce = (unsigned)((P.M + blockDim.x - 1) / blockDim.x);
    for (unsigned t; (t = take(c + kForceTake)) < nforce;) {
        const int64_t j = (int64_t)t * blockDim.x + threadIdx.x;
        if (j < P.M) P.gforce[j] = forcing(P, n, j);
        finish(c + kForceDone);
    }
}

// The history pipeline as units handed out by counters: columns, then row pairs, then inverse
// columns, then chunks of interpolation points, each phase starting once every unit of the one
// before is done; last, the FIR tail of the next step (any time before the step ends).  Any number
// of blocks may take part, at any time; false if a wait ran out.
__device__ __forceinline__ bool history_units(const DevPlan& P, int64_t n, unsigned char* smraw) {
    unsigned* c = P.bar;
    double2* Y = (double2*)P.work;
    double2* T = (double2*)P.spec;
    const unsigned ncols = (unsigned)P.L2, nrows = (unsigned)(P.L1 / 2 + 1);
    const unsigned nint = (unsigned)((P.M + P.R + blockDim.x - 1) / blockDim.x);
    const unsigned nforce = (unsigned)((P.M + blockDim.x - 1) / blockDim.x);
    const unsigned ntail = (unsigned)((P.K + 1 + kTailModes - 1) / kTailModes);
    unsigned first = ncols;
    for (unsigned t; (t = take(c + kColTake)) < ncols;) {
        cols_phase(P, n, Y, (int)t, smraw);
        finish(c + kColDone);
        first = min(first, t);
    }
    // each column is taken once, so the first column a block took ranks it among the prefetchers
    if (first < ncols)
        prefetch_step_state(P, (int64_t)first * blockDim.x + threadIdx.x, (int64_t)ncols * blockDim.x);
    if (!wait_for(P, c + kColDone, ncols)) return false;
    for (unsigned t; (t = take(c + kRowTake)) < nrows;) {
        rows_phase(P, n, Y, T, (int)t, 1, smraw);
        finish(c + kRowDone);
    }
    if (!wait_for(P, c + kRowDone, nrows)) return false;
    for (unsigned t; (t = take(c + kIcolTake)) < ncols;) {
        icols_phase(P, T, (int)t, smraw);
        finish(c + kIcolDone);
    }
    forcing_units(P, n);
    if (!wait_for(P, c + kIcolDone, ncols)) return false;
    if (!wait_for(P, c + kForceDone, nforce)) return false;
    for (unsigned t; (t = take(c + kIntTake)) < nint;)
        interp_points(P, n, (int64_t)t * blockDim.x + threadIdx.x, P.M + P.R, P.gforce);
    for (unsigned t; (t = take(c + kTailTake)) < ntail;) fir_tail(P, n, (int)t * kTailModes);
    return true;
}

__global__ void __launch_bounds__(kStepThreads, 4) k_step(DevPlan P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ bool last;
    const int64_t n = load_step(P);
    const int G = gridDim.x, b = blockIdx.x;
    unsigned* c = P.bar;
    // blocks [0, hist_blocks) start with the history pipeline, the rest with the local sum;
    // whoever runs out of its first kind of work helps with the other
    const bool hist_first = b < P.hist_blocks;
    if (hist_first && !history_units(P, n, smraw)) return;
    if (!hist_first) forcing_units(P, n);
    local_items_loop(P, n);
    if (!hist_first && !history_units(P, n, smraw)) return;
    // grid barrier: every item partial and right-hand side of the step is stored
    finish(c + kGrid);
    if (!wait_for(P, c + kGrid, (unsigned)G)) return;
    const int nw = blockDim.x >> 5;
    solve_blocks(P, n, (int64_t)b * nw + (threadIdx.x >> 5), (int64_t)G * nw,
                 (double*)smraw + (threadIdx.x >> 5) * kSolveStage);
    // the block that finishes last (every other block has stored its densities and is past every
    // wait) resets the counters, reads out the receivers and advances the step counter
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long done = atomicAdd((unsigned long long*)&P.step[1], 1ull);
        last = (done == (unsigned long long)G - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNumCounters; i++) c[i] = 0u;
        *P.item_ctr = 0ull;
    }
    receivers_readout(P, n);
    __syncthreads();
    if (threadIdx.x == 0) {
        P.step[1] = 0;
        __threadfence();
        P.step[0] = n + 1;
    }
}

}  // namespace wave1d
