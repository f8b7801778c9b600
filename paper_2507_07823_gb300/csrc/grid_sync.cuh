// Bounded waits between the blocks of a one-launch (cooperative) step: counters in device memory
// that blocks increment when a unit of work is done (finish) and poll until a phase is complete
// (wait_for, wait_for2).  Every wait gives up after DevPlan.spin_limit polls, latching
// WAVE1D_ETIMEOUT in the status word; the other blocks then give up at their next wait.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "../../include/wave1d.h"

namespace wave1d {

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
            if (++polls > P.spin_limit) {
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

// thread 0 waits until *a >= ta and *b >= tb (one poll reads both)
__device__ __forceinline__ bool wait_for2(const DevPlan& P, const unsigned* a, unsigned ta, const unsigned* b,
                                          unsigned tb) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        unsigned polls = 0;
        for (;;) {
            const unsigned va = ld_acquire(a), vb = ld_acquire(b);
            if (va >= ta && vb >= tb) break;
            if (++polls > P.spin_limit) {
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

// the block's writes of a finished unit become visible before the unit is counted
__device__ __forceinline__ void finish(unsigned* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

}  // namespace wave1d
