// One ordinary time step n -> n+1 of the WFP march as a single cooperative launch.
//
// The step has two independent halves that both start from sigma^{<= n}: the local explicit sum
// (Sec. 4.1), which streams the stored weights and is bound by HBM, and the history pipeline
// (Sec. 3: type-1 NUFFT, mode update, type-2 NUFFT, interpolation), a chain of short latency-bound
// passes.  As separate launches they run back to back, each short pass paying a launch and a
// ramp.  Here both run at once:
//
//   blocks [0, H)   the history pipeline: block h runs column h, row pair h, inverse column h and
//                   interpolation chunks h, h + H, ..., each phase waiting (on a counter) for the
//                   one before; then local sum items
//   blocks [H, G)   the prologue (the FIR tail and the forcing of the step, which need nothing
//                   computed in it), then local sum items (atomic counter)
//   all blocks      grid barrier; block solve of eq. linearSystem; the block that finishes last
//                   resets the counters, reads out the receivers and advances the step counter
//
// The history blocks are consecutive block indices, which the hardware spreads over different
// SMs: their FP64 work (GB300 issues one FP64 warp instruction per 64 cycles per SM partition)
// then uses many SMs' FP64 units, which the local sum (FP32 and loads) leaves idle; the prologue's
// FP64 is spread over all the other blocks.  Units are assigned, not taken from counters, because
// every atomic round trip costs microseconds while HBM is saturated.  Every block is resident (the
// launch is cooperative) and every wait is bounded: a wait that runs out latches WAVE1D_ETIMEOUT in
// the status word and the block returns; the other blocks then give up at their next wait.
// Projection steps (Sec. 4.4) use the per-stage kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "grid_sync.cuh"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {


// counters in P.bar (all zero between steps)
enum : int { kColDone = 0, kRowDone, kIcolDone, kTailDone, kForceDone, kGrid, kNumCounters };

// The small working set of the later phases on the critical path (per-mode factors and FIR
// tails, interpolation kernels, solve groups and block inverses: a few MB) is pulled into L2 after
// the column pass, so the latency-bound phases that follow find it there.
__device__ __forceinline__ void prefetch_step_state(const DevPlan& P, int64_t tid, int64_t nt) {
    const size_t K1 = (size_t)P.K + 1, M = (size_t)P.M, R = (size_t)P.R, w = (size_t)P.w;
    prefetch_l2(P.twiddle, (size_t)P.L * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.pq, K1 * 2 * sizeof(double), tid, nt);              // taps m = 0
    prefetch_l2(P.ftail, K1 * 4 * sizeof(double), tid, nt);
    prefetch_l2(P.modefac, K1 * 8 * sizeof(double), tid, nt);
    prefetch_l2(P.rot, K1 * 3 * sizeof(double), tid, nt);
    prefetch_l2(P.alpha, K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.alpha_p, K1 * 2 * sizeof(double), tid, nt);
    prefetch_l2(P.sp_i0, M * sizeof(int32_t), tid, nt);
    prefetch_l2(P.sp_ker, M * w * sizeof(double), tid, nt);
    prefetch_l2(P.beta, M * sizeof(double), tid, nt);
    if (R) {
        prefetch_l2(P.rc_i0, R * sizeof(int32_t), tid, nt);
        prefetch_l2(P.rc_ker, R * w * sizeof(double), tid, nt);
    }
    const size_t ng = (size_t)P.n_sgroups;
    prefetch_l2(P.sg_j, ng * 32 * sizeof(int32_t), tid, nt);
    prefetch_l2(P.sg_meta, ng * 32 * sizeof(int32_t), tid, nt);
    prefetch_l2(P.sg_off, ng * 32 * sizeof(int64_t), tid, nt);
    prefetch_l2(P.sg_beta, ng * 32 * sizeof(double), tid, nt);
    prefetch_l2(P.sg_ip, ng * 32 * sizeof(int64_t), tid, nt);
    prefetch_l2(P.sg_icnt, ng * 32 * sizeof(int32_t), tid, nt);
    prefetch_l2(P.inv, (size_t)P.inv_len * sizeof(double), tid, nt);
}

// Work of the step that needs nothing computed in it, split over the blocks that start with the
// local sum (rank r of nl): the FIR tail (taps m >= 1, which read only S^{< n}) of modes
// [r mp, (r + 1) mp), an octet of lanes per mode, and the forcing g_j(t_{n+1}) of springs
// j = r, r + nl, ... (strided, so the springs near the pulses, whose FP64 exponentials dominate,
// spread over all blocks).  Warp w takes chunks w, w + 8, ... (four modes or 32 springs each) and
// counts the modes / springs it finished, so the waits need no block count.
__device__ __forceinline__ void prologue(const DevPlan& P, int64_t n, int r, int nl) {
    unsigned* c = P.bar;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int K1 = P.K + 1;
    const int mp = (K1 + nl - 1) / nl;
    const int mine = max(0, min(mp, K1 - r * mp));             // modes of this block
    const int64_t ms = r < P.M ? (P.M - r + nl - 1) / nl : 0;  // springs of this block
    const int nT = (mine + 3) / 4;
    const int nF = (int)((ms + 31) / 32);
    for (int ch = wid; ch < nT + nF; ch += nw) {
        unsigned cnt;
        unsigned* ctr;
        if (ch < nT) {
            const int loc = ch * 4 + (lane >> 3);
            fir_tail(P, n, r * mp + loc, loc < mine);
            cnt = (unsigned)min(4, mine - ch * 4);
            ctr = c + kTailDone;
        } else {
            const int64_t i = (int64_t)(ch - nT) * 32 + lane;
            const int64_t j = r + (int64_t)nl * i;
            if (i < ms) P.gforce[j] = forcing(P, n, j);
            cnt = (unsigned)min((int64_t)32, ms - (int64_t)(ch - nT) * 32);
            ctr = c + kForceDone;
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(ctr, cnt);
        }
    }
}

// The history pipeline on blocks h = 0 .. H-1 (H = hist_blocks, all resident): columns, row pairs
// and inverse columns h, h + H, ..., then interpolation chunks h, h + H, ...; each phase starts
// once every unit of the one before is counted done (the rows also wait for the FIR tail, the
// interpolation for the forcing).  False if a wait ran out.
__device__ __forceinline__ bool history_blocks(const DevPlan& P, int64_t n, int h, unsigned char* smraw) {
    unsigned* c = P.bar;
    double2* Y = (double2*)P.work;
    double2* T = (double2*)P.spec;
    const int H = P.hist_blocks;
    const int ncols = P.L2, nrows = P.L1 / 2 + 1;
    const int64_t nint = (P.M + P.R + kInterpPoints - 1) / kInterpPoints;
    for (int t = h; t < ncols; t += H) {
        cols_phase(P, n, Y, t, smraw);
        if (P.hold_unit && t == 0) continue;       // fault injection: unit 0 is never counted
        finish(c + kColDone);
    }
    prefetch_step_state(P, (int64_t)h * blockDim.x + threadIdx.x, (int64_t)H * blockDim.x);
    if (!wait_for2(P, c + kColDone, (unsigned)ncols, c + kTailDone, (unsigned)(P.K + 1))) return false;
    for (int t = h; t < nrows; t += H) {
        rows_phase(P, n, Y, T, t, 1, smraw);
        finish(c + kRowDone);
    }
    if (!wait_for(P, c + kRowDone, (unsigned)nrows)) return false;
    for (int t = h; t < ncols; t += H) {
        icols_phase(P, T, t, smraw);
        finish(c + kIcolDone);
    }
    if (!wait_for2(P, c + kIcolDone, (unsigned)ncols, c + kForceDone, (unsigned)P.M)) return false;
    for (int64_t t = h; t < nint; t += H) interp_chunk(P, n, t, P.gforce);
    return true;
}

__global__ void __launch_bounds__(kStepThreads, 4) k_step(DevPlan P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ bool last;
    const int64_t n = load_step(P);
    const int G = gridDim.x, b = blockIdx.x;
    unsigned* c = P.bar;
    // blocks [0, hist_blocks) run the history pipeline, the others the prologue; then everyone
    // takes local sum items
    if (b < P.hist_blocks) {
        if (!history_blocks(P, n, b, smraw)) return;
    } else {
        prologue(P, n, b - P.hist_blocks, G - P.hist_blocks);
    }
    local_items_loop(P, n);
    // grid barrier: every item partial and right-hand side of the step is stored
    finish(c + kGrid);
    if (!wait_for(P, c + kGrid, (unsigned)G)) return;
    // solve tasks interleaved over the blocks (task t on block t mod G), so the few hundred
    // tasks' FP64 work spreads over every SM instead of queueing on the first blocks' FP64 units
    const int nw = blockDim.x >> 5;
    solve_tasks(P, n, (int64_t)(threadIdx.x >> 5) * G + b, (int64_t)G * nw,
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
