// Batched march: many independent periodic instances (own springs, stiffnesses, incident pulse
// and receivers) sharing dt, N_t, tol and p advance together, one pass of launches per step over
// all of them (declared in include/wave1d.h).
//
// The instances' tables are joined (batch_host.cpp): the local sum (Sec. 4.1) and the block solve
// (eq. linearSystem) run as the one-plan per-stage kernels over the joined items and solve groups,
// with the density rings in instance-major spring order.  The history part (Sec. 3) is per
// instance: its spreading and interpolation (eqs. densco, historySol1) run through a batched
// NUFFT plan (one launch per pass over all instances, instance-major fine grids), and the FFT
// passes, the FIR driving terms and the mode update run as the one-plan phases with one grid row
// per instance, each instance reading its own view of the plan (its modes, S ring, FIR tail, FFT
// buffers and fine grid).  Every launch reads the step index from the device counter, so one step
// is captured once in a CUDA graph and replayed.
//
// Instances too large or too dense for stored weights are not joined: each is a plan of its own
// without pair lists (range.cu), and the step graph holds its ordinary step as one branch (its
// private stream forked after the joined instances' step and joined before the graph's end,
// plan_hooks.h), so those instances run concurrently with one another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "batch_host.h"
#include "internal.h"
#include "plan_hooks.h"
#include "grid_sync.cuh"
#include "nufft_units.cuh"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {
__global__ void k_local_items(DevPlan P);
__global__ void k_solve(DevPlan P);
__global__ void k_mx_gather(DevPlan P, const int64_t* perm, double* c);
__global__ void k_mx_receivers(int64_t R, const int64_t* perm, const double* u, double* uHr);

// forward FFT column pass of one instance's fine grid: for column i2, FFT over i1 of
// z[i2 + L2 i1] (sign +), times e^{+2 pi i i2 k1 / L}  ->  Y[k1 L2 + i2]; sm: L1 + L1/2 points
__device__ __forceinline__ void bfft_col(const double2* __restrict__ in, double2* __restrict__ out,
                                         const double2* __restrict__ tw, int L, int L1, int L2, int logL1, int i2,
                                         double2* sm) {
    double2* twN = sm + L1;
    for (int j = threadIdx.x; j < L1 / 2; j += blockDim.x) twN[j] = tw[j * (L / L1)];
    for (int i1 = threadIdx.x; i1 < L1; i1 += blockDim.x) sm[__brev(i1) >> (32 - logL1)] = in[i2 + (int64_t)L2 * i1];
    __syncthreads();
    fft_lines(sm, nullptr, twN, L1, logL1);
    for (int k1 = threadIdx.x; k1 < L1; k1 += blockDim.x)
        out[(int64_t)k1 * L2 + i2] = cmul(sm[k1], tw[((int64_t)i2 * k1) & (L - 1)]);
}

// the column pass of every instance's fine grid (blockIdx.y = instance)
__global__ void k_bfft_cols(const double2* __restrict__ grids, double2* __restrict__ Ys,
                            const double2* __restrict__ tw, int L, int L1, int L2, int logL1) {
    extern __shared__ double2 sm[];
    bfft_col(grids + (int64_t)blockIdx.y * L, Ys + (int64_t)blockIdx.y * L, tw, L, L1, L2, logL1, blockIdx.x, sm);
}

// FIR tails, rows (FFT + mode update + first inverse pass) and inverse columns of every
// instance: the one-plan phases on the instance's view (blockIdx.y = instance)
__global__ void k_bhist_tail(const DevPlan* __restrict__ views) {
    const DevPlan& P = views[blockIdx.y];
    const int k = blockIdx.x * kTailModes + (int)(threadIdx.x >> 3);
    fir_tail(P, load_step(P), k, k <= P.K);
}

__global__ void k_bhist_rows(const DevPlan* __restrict__ views) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const DevPlan& P = views[blockIdx.y];
    rows_phase(P, load_step(P), (const double2*)P.work, (double2*)P.spec, blockIdx.x, 1, smraw);
}

__global__ void k_bhist_icols(const DevPlan* __restrict__ views) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const DevPlan& P = views[blockIdx.y];
    icols_phase(P, (const double2*)P.spec, blockIdx.x, smraw);
}

// u_H at spring perm[i] and the right-hand side rhs_j = -g_j(t_{n+1}) - beta_j u_H(x_j) with the
// incident wave of the spring's instance: g_j = beta_j f_b(x_j - t), f_b one Gaussian periodised
// over 2 pi (eq. gj; the same sum, with the same 12-width cut, as the one-plan forcing)
__device__ __forceinline__ void b_rhs_point(const DevPlan& P, int64_t n, int64_t i, const int64_t* __restrict__ perm,
                                            const double* __restrict__ u, const int32_t* __restrict__ inst_of,
                                            const double* __restrict__ pulse) {
    const double kTwoPi = 6.283185307179586476925286766559;
    const double kInvTwoPi = 0.15915494309189533576888376337251;
    const double t = (double)(n + 1) * P.dt;
    const int64_t j = perm[i];
    const double* pl = pulse + 3 * (int64_t)inst_of[j];
    const double amp = pl[0], cen = pl[1], iw = pl[2];
    const double s = P.x[j] - t, span = 12.0 / iw;
    const int64_t m0 = (int64_t)floor((cen - s - span) * kInvTwoPi);
    const int64_t m1 = (int64_t)ceil((cen - s + span) * kInvTwoPi);
    double f = 0.0;
    for (int64_t m = m0; m <= m1; m++) {
        const double z = (s + kTwoPi * (double)m - cen) * iw;
        if (fabs(z) <= 12.0) f += amp * exp(-0.5 * z * z);
    }
    const double uh = u[i], bj = P.beta[j];
    P.uH[j] = uh;
    P.rhs[j] = -bj * f - bj * uh;
}

__global__ void k_b_rhs(DevPlan P, const int64_t* __restrict__ perm, const double* __restrict__ u,
                        const int32_t* __restrict__ inst_of, const double* __restrict__ pulse) {
    const int64_t n = load_step(P);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M; i += (int64_t)gridDim.x * blockDim.x)
        b_rhs_point(P, n, i, perm, u, inst_of, pulse);
}

// ---------------------------------------------------------------------------------------------
// The batched step as one cooperative launch (all blocks resident), the persistent form of the
// per-pass launches of enqueue_batch_step with the same unit bodies and sums, so both give the
// same bits:
//   blocks [0, H)   the history chain of every instance: FP64 spreading (one NUFFT range per
//                   unit), FFT columns (instance, column), row pairs (instance, row pair: FFT,
//                   mode update, first inverse pass), inverse columns, then interpolation tiles
//                   of the springs (each followed by their right-hand sides) and of the receivers;
//                   each phase waits for the one before; then local-sum items
//   blocks [H, G)   the prologue (sigma^n gathered into the NUFFT's point order, the FIR tails of
//                   every instance's modes: both read only earlier steps), then local-sum items
//   all blocks      grid barrier; block solve; the block that finishes last resets the counters,
//                   reads out the receivers and advances the step counter
// Every wait is bounded (DevPlan.spin_limit): one that runs out latches WAVE1D_ETIMEOUT.
// ---------------------------------------------------------------------------------------------
enum : int { kBGather = 0, kBTail, kBSpread, kBCol, kBRow, kBIcol, kBGrid, kBNumCounters };
constexpr int kBStepThreads = 256;

struct BatchStep {
    DevPlan g;                  // joined view (local sum, solve, receivers), sig_hist set per graph
    const DevPlan* views;       // per instance (history phases)
    int B, H;                   // instances, history blocks
    NuDev64 ns, nr;             // NUFFT of the springs and of the receivers (nr.M = 0: none)
    const int64_t *perm_s, *perm_r;
    const int32_t* inst_of;
    const double* pulse;
    double *c, *u, *ur;
    unsigned* bar;              // kBNumCounters counters, zero between steps
};

template <int W>
__global__ void __launch_bounds__(kBStepThreads, 4) k_batch_step(BatchStep A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ bool last;
    const DevPlan& P = A.g;
    const int64_t n = load_step(P);
    const int G = gridDim.x, b = blockIdx.x, H = A.H;
    unsigned* c = A.bar;
    const int L = P.L, L1 = P.L1, L2 = P.L2, nrows = P.L1 / 2 + 1, K1 = P.K + 1;
    const int64_t ngather = (A.ns.M + kBStepThreads - 1) / kBStepThreads;
    const int ntail = (K1 + kTailModes - 1) / kTailModes;
    if (b < H) {
        const DevPlan* V = A.views;
        // spreading of sigma^n (gathered by the prologue) onto every instance's fine grid
        if (!wait_for(P, c + kBGather, (unsigned)ngather)) return;
        for (int64_t t = b; t < A.ns.nunits; t += H) {
            spread64_unit<W>(A.ns.ranges[t], A.ns.runs, A.c, A.ns.ker, (double*)V[0].grid,
                             (double(*)[W])smraw, (int*)(smraw + (size_t)(kRangeCells64 + 16) * W * sizeof(double)));
            finish(c + kBSpread);
        }
        if (!wait_for(P, c + kBSpread, (unsigned)A.ns.nunits)) return;
        const int logL1 = 31 - __clz(L1);
        for (int64_t t = b; t < (int64_t)A.B * L2; t += H) {
            const int ib = (int)(t / L2), i2 = (int)(t % L2);
            __syncthreads();
            bfft_col((const double2*)V[ib].grid, (double2*)V[ib].work, (const double2*)P.twiddle, L, L1, L2, logL1, i2,
                     (double2*)smraw);
            finish(c + kBCol);
        }
        if (!wait_for2(P, c + kBCol, (unsigned)(A.B * L2), c + kBTail, (unsigned)(A.B * ntail))) return;
        for (int64_t t = b; t < (int64_t)A.B * nrows; t += H) {
            const int ib = (int)(t / nrows), k1 = (int)(t % nrows);
            __syncthreads();
            rows_phase(V[ib], n, (const double2*)V[ib].work, (double2*)V[ib].spec, k1, 1, smraw);
            finish(c + kBRow);
        }
        if (!wait_for(P, c + kBRow, (unsigned)(A.B * nrows))) return;
        for (int64_t t = b; t < (int64_t)A.B * L2; t += H) {
            const int ib = (int)(t / L2), i2 = (int)(t % L2);
            __syncthreads();
            icols_phase(V[ib], (const double2*)V[ib].spec, i2, smraw);
            finish(c + kBIcol);
        }
        if (!wait_for(P, c + kBIcol, (unsigned)(A.B * L2))) return;
        // interpolation tiles: the springs' (then their right-hand sides, point by point in the
        // thread that interpolated it) and the receivers' (then their u_H)
        const int64_t ts = (A.ns.M + kInterpTile - 1) / kInterpTile, tr = (A.nr.M + kInterpTile - 1) / kInterpTile;
        for (int64_t t = b; t < ts + tr; t += H) {
            if (t < ts) {
                interp64_unit(t, (const double*)V[0].grid, A.u, A.ns.i0, A.ns.ker, A.ns.M, A.ns.w, A.ns.nf,
                              (double*)smraw);
                const int64_t i = t * kInterpTile + threadIdx.x;
                if (threadIdx.x < kInterpTile && i < A.ns.M) b_rhs_point(P, n, i, A.perm_s, A.u, A.inst_of, A.pulse);
            } else {
                const int64_t tt = t - ts;
                interp64_unit(tt, (const double*)V[0].grid, A.ur, A.nr.i0, A.nr.ker, A.nr.M, A.nr.w, A.nr.nf,
                              (double*)smraw);
                const int64_t i = tt * kInterpTile + threadIdx.x;
                if (threadIdx.x < kInterpTile && i < A.nr.M) P.uHr[A.perm_r[i]] = A.ur[i];
            }
        }
    } else {
        // prologue on blocks H .. G - 1 (rank r of nl): gather chunks, then FIR-tail units
        const int r = b - H, nl = G - H;
        const double* sg = P.sig + (int64_t)ring_slot(n, P.ring) * P.M;
        for (int64_t t = r; t < ngather; t += nl) {
            const int64_t i = t * kBStepThreads + threadIdx.x;
            if (i < A.ns.M) A.c[i] = sg[A.perm_s[i]];
            finish(c + kBGather);
        }
        for (int64_t t = r; t < (int64_t)A.B * ntail; t += nl) {
            const int ib = (int)(t / ntail), ch = (int)(t % ntail);
            const int k = ch * kTailModes + (int)(threadIdx.x >> 3);
            fir_tail(A.views[ib], n, k, k <= P.K);
            finish(c + kBTail);
        }
    }
    local_items_loop(P, n);
    // grid barrier: every item partial and right-hand side of the step is stored
    finish(c + kBGrid);
    if (!wait_for(P, c + kBGrid, (unsigned)G)) return;
    const int nw = blockDim.x >> 5;
    solve_tasks(P, n, (int64_t)(threadIdx.x >> 5) * G + b, (int64_t)G * nw, (double*)smraw + (threadIdx.x >> 5) * kSolveStage);
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
        for (int i = 0; i < kBNumCounters; i++) c[i] = 0u;
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

using namespace wave1d;

namespace {
thread_local std::string g_batch_error;

int bfail(int code, const std::string& msg) {
    g_batch_error = msg;
    return code;
}

#define BCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bfail(WAVE1D_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)
}  // namespace

struct wave1d_batch_s {
    BatchTables bt;
    DevPlan g{};                       // joined view: local sum, solve, receivers
    DevPlan* d_views = nullptr;        // one view per instance for the history phases
    std::vector<void*> allocs;
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    int device = 0, sms = 1, B = 0, chunk = 32;
    int64_t n = 0;
    wave1d_nufft_t nu_s = nullptr, nu_r = nullptr;
    int64_t *perm_s = nullptr, *perm_r = nullptr;
    int32_t* inst_of = nullptr;
    double *pulse = nullptr, *c = nullptr, *u = nullptr, *ur = nullptr, *grids = nullptr, *work = nullptr,
           *sig_hist = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step without / with the density history
    // the one-launch step (k_batch_step): used when the kernel width has an instance and the
    // device launches cooperative grids (opts.step_kernel)
    bool persist = false;
    int W = 0, H = 0;
    unsigned pgrid = 0;
    size_t psmem = 0;
    unsigned* bar = nullptr;
    NuDev64 ns{}, nr{};
    // all instances: springs and receivers (instance-major), steps planned, form of each instance
    // (0: joined tables above, 1: its own plan without pair lists)
    int n_inst = 0;
    int64_t M_all = 0, R_all = 0, Nt = 0;
    std::vector<int> form;
    bool has_joined = false;
    // the instances without pair lists: their plans, stepped as branches of the step graph
    std::vector<wave1d_plan_t> sub;
    std::vector<PlanHooks> sub_hooks;
    std::vector<double*> sub_sig;
    std::vector<int64_t> sub_moff, sub_roff;          // their first spring and receiver overall
    // copies of the joined rings' columns to the output rows: (joined column, output column, width)
    std::vector<int64_t> seg_m, seg_r;
};

namespace {

template <typename T>
int balloc(wave1d_batch_t p, T** out, size_t count) {
    *out = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return bfail(WAVE1D_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    p->allocs.push_back(q);
    *out = (T*)q;
    BCK(cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), p->s));
    return WAVE1D_OK;
}

template <typename T>
int bupload(wave1d_batch_t p, const std::vector<T>& v, T** out) {
    int rc = balloc(p, out, v.size());
    if (rc || v.empty()) return rc;
    BCK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p->s));
    return WAVE1D_OK;
}

template <typename T>
int bup(wave1d_batch_t p, const std::vector<T>& v, const T** field) {
    T* q;
    int rc = bupload(p, v, &q);
    *field = q;
    return rc;
}

// the joined tables on the device: what k_local_items, k_solve and the receivers' readout read
int upload_joined(wave1d_batch_t p) {
    const HostPlan& h = p->bt.g;
    const Params& P = h.P;
    DevPlan& d = p->g;
    d.M = P.M;
    d.R = P.R;
    d.K = P.K;
    d.W = P.W;
    d.m_max = P.m_max;
    d.ring = P.ring;
    d.nf = P.nf;
    d.L = P.L;
    d.L1 = P.L1;
    d.L2 = P.L2;
    d.w = P.nufft_w;
    d.bc = P.bc;
    d.dt = P.dt;
    d.chunk = p->chunk;
    int rc;
    int64_t* i64;
    double* f64;
    unsigned long long* ctr;
    if ((rc = balloc(p, &i64, 2))) return rc;
    d.step = i64;
    if ((rc = balloc(p, &ctr, 1))) return rc;
    d.item_ctr = ctr;
    int* st;
    if ((rc = balloc(p, &st, 1))) return rc;
    d.status = st;
    if ((rc = bup(p, h.x, &d.x)) || (rc = bup(p, h.beta, &d.beta)) || (rc = bup(p, h.perm, &d.perm)) ||
        (rc = bup(p, h.pq, &d.pq)) || (rc = bup(p, h.rot, &d.rot)) || (rc = bup(p, h.twiddle, &d.twiddle)) ||
        (rc = bup(p, h.modefac, &d.modefac)) || (rc = bup(p, h.deconv1, &d.deconv1)) ||
        (rc = bup(p, h.deconv2, &d.deconv2)))
        return rc;
    if ((rc = balloc(p, &f64, (size_t)P.M))) return rc;
    d.rhs = f64;
    if ((rc = balloc(p, &f64, (size_t)P.M))) return rc;
    d.uH = f64;
    if ((rc = balloc(p, &f64, (size_t)P.M))) return rc;
    d.clocal = f64;
    if ((rc = balloc(p, &f64, (size_t)P.M * P.ring))) return rc;
    d.sig = f64;
    float* f32;
    if ((rc = balloc(p, &f32, (size_t)P.M * P.ring * 4))) return rc;
    d.sig2 = f32;
    // local-sum items of the springs and of the receivers
    const LocalItems& L = h.litems;
    const LocalItems& Rr = h.ritems;
    d.l_mfirst = L.m_first;
    d.r_mfirst = Rr.m_first;
    d.l_nitems = (int64_t)L.row.size();
    d.r_nitems = (int64_t)Rr.row.size();
    if ((rc = bup(p, L.item_ptr, &d.l_item_ptr)) || (rc = bup(p, L.row, &d.l_row)) || (rc = bup(p, L.s0, &d.l_s0)) ||
        (rc = bup(p, L.len, &d.l_len)) || (rc = bup(p, L.wbase, &d.l_wbase)) || (rc = bup(p, L.src, &d.l_src)) ||
        (rc = bup(p, L.w, &d.l_w)) || (rc = bup(p, Rr.item_ptr, &d.r_item_ptr)) || (rc = bup(p, Rr.s0, &d.r_s0)) ||
        (rc = bup(p, Rr.len, &d.r_len)) || (rc = bup(p, Rr.wbase, &d.r_wbase)) || (rc = bup(p, Rr.src, &d.r_src)) ||
        (rc = bup(p, Rr.w, &d.r_w)))
        return rc;
    if ((rc = balloc(p, &f64, (size_t)std::max<int64_t>(1, d.l_nitems)))) return rc;
    d.l_part = f64;
    if ((rc = balloc(p, &f64, (size_t)std::max<int64_t>(1, d.r_nitems)))) return rc;
    d.r_part = f64;
    {
        const int64_t NL = d.l_nitems, NR = d.r_nitems;
        std::vector<int32_t> order((size_t)(NL + NR));
        auto len = [&](int32_t o) { return o < NL ? L.len[o] : Rr.len[o - NL]; };
        for (int64_t i = 0; i < NL + NR; i++) order[i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
        if ((rc = bup(p, order, &d.item_order))) return rc;
    }
    // receivers' m = 0 terms, padded to whole warps
    int64_t most = 0;
    for (int64_t r = 0; r < P.R; r++) most = std::max(most, h.r0_ptr[r + 1] - h.r0_ptr[r]);
    d.r0_stride = (int)((most + 31) / 32 * 32);
    std::vector<int32_t> psrc((size_t)P.R * d.r0_stride, 0);
    std::vector<double> pw((size_t)P.R * d.r0_stride, 0.0);
    for (int64_t r = 0; r < P.R; r++)
        for (int64_t e = h.r0_ptr[r]; e < h.r0_ptr[r + 1]; e++) {
            psrc[(size_t)r * d.r0_stride + (e - h.r0_ptr[r])] = h.r0_src[e];
            pw[(size_t)r * d.r0_stride + (e - h.r0_ptr[r])] = h.r0_w[e];
        }
    if ((rc = bup(p, psrc, &d.r0p_src)) || (rc = bup(p, pw, &d.r0p_w))) return rc;
    if ((rc = balloc(p, &f64, (size_t)std::max<int64_t>(1, P.R)))) return rc;
    d.uHr = f64;
    if ((rc = balloc(p, &f64, (size_t)p->chunk * std::max<int64_t>(1, P.R)))) return rc;
    d.rec_hist = f64;
    // blocks and solve groups
    if ((rc = bup(p, h.blk_ptr, &d.blk_ptr)) || (rc = bup(p, h.blk_members, &d.blk_members)) ||
        (rc = bup(p, h.blk_inv_off, &d.blk_inv_off)) || (rc = bup(p, h.inv, &d.inv)) ||
        (rc = bup(p, h.sg_j, &d.sg_j)) || (rc = bup(p, h.sg_meta, &d.sg_meta)) || (rc = bup(p, h.sg_off, &d.sg_off)) ||
        (rc = bup(p, h.sg_beta, &d.sg_beta)) || (rc = bup(p, h.sg_ip, &d.sg_ip)) || (rc = bup(p, h.sg_icnt, &d.sg_icnt)) ||
        (rc = bup(p, h.sg_smax, &d.sg_smax)) || (rc = bup(p, h.big_blk, &d.big_blk)) ||
        (rc = bup(p, h.big_row0, &d.big_row0)))
        return rc;
    d.nblocks = (int64_t)h.blk_ptr.size() - 1;
    d.n_sgroups = (int64_t)h.sg_smax.size();
    d.n_big = (int64_t)h.big_blk.size();
    d.inv_len = (int64_t)h.inv.size();
    return WAVE1D_OK;
}

// one view of the plan per instance: its modes, S ring, FIR tail, FFT buffers and fine grid
int upload_views(wave1d_batch_t p) {
    const Params& P = p->bt.g.P;
    const int64_t B = p->B, K1 = P.K + 1;
    double *alpha, *alpha_p, *Sring, *ftail, *spec, *spec2;
    int rc;
    if ((rc = balloc(p, &alpha, (size_t)B * 2 * K1)) || (rc = balloc(p, &alpha_p, (size_t)B * 2 * K1)) ||
        (rc = balloc(p, &Sring, (size_t)B * P.W * 2 * K1)) || (rc = balloc(p, &ftail, (size_t)B * 4 * K1)) ||
        (rc = balloc(p, &p->work, (size_t)B * 2 * P.L)) || (rc = balloc(p, &spec, (size_t)B * 2 * P.L)) ||
        (rc = balloc(p, &spec2, (size_t)B * 2 * P.L)) || (rc = balloc(p, &p->grids, (size_t)B * P.nf)))
        return rc;
    std::vector<DevPlan> views((size_t)B, p->g);
    for (int64_t b = 0; b < B; b++) {
        DevPlan& v = views[b];
        v.alpha = alpha + b * 2 * K1;
        v.alpha_p = alpha_p + b * 2 * K1;
        v.Sring = Sring + b * P.W * 2 * K1;
        v.ftail = ftail + b * 4 * K1;
        v.work = p->work + b * 2 * P.L;
        v.spec = spec + b * 2 * P.L;
        v.spec2 = spec2 + b * 2 * P.L;
        v.grid = p->grids + b * P.nf;
    }
    return bupload(p, views, &p->d_views);
}

// kernel widths the one-launch batched step is built for (tol 1e-6 .. 1e-13); others take the
// per-pass launches
constexpr int kBStepWMin = 7, kBStepWMax = 14;

template <int W>
const void* batch_step_fn() {
    return (const void*)k_batch_step<W>;
}

const void* batch_step_kernel(int w) {
    switch (w) {
        case 7: return batch_step_fn<7>();
        case 8: return batch_step_fn<8>();
        case 9: return batch_step_fn<9>();
        case 10: return batch_step_fn<10>();
        case 11: return batch_step_fn<11>();
        case 12: return batch_step_fn<12>();
        case 13: return batch_step_fn<13>();
        case 14: return batch_step_fn<14>();
        default: return nullptr;
    }
}

// size the one-launch step: shared memory of its largest unit, as many blocks as are resident, the
// history group one block per unit of its widest phase, at most half the blocks
int setup_batch_step(wave1d_batch_t p, const wave1d_opts& o) {
    const Params& P = p->bt.g.P;
    p->persist = false;
    if (!o.step_kernel) return WAVE1D_OK;
    if (nufft_dev64(p->nu_s, p->ns) != WAVE1D_OK) return WAVE1D_OK;
    if (P.R > 0 && nufft_dev64(p->nu_r, p->nr) != WAVE1D_OK) return WAVE1D_OK;
    if (P.R == 0) p->nr = NuDev64{nullptr, nullptr, 0, nullptr, nullptr, 0, p->ns.w, p->ns.nf};
    const int w = p->ns.w;
    const void* fn = batch_step_kernel(w);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device);
    if (!fn || !coop) return WAVE1D_OK;
    const size_t spread = (size_t)(kRangeCells64 + 16) * w * sizeof(double) + (size_t)(kSpread64Runs + 1) * sizeof(int);
    const size_t sm = std::max({spread, kInterp64Smem, fft_smem_bytes(P.L1), rows_phase_smem(P.L2),
                                icols_phase_smem(P.L1), (size_t)kSolveStage * sizeof(double) * (kBStepThreads / 32)});
    int occ = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBStepThreads, sm) != cudaSuccess)
        return bfail(WAVE1D_ECUDA, "cannot configure the batched step kernel");
    if (occ < 1) return WAVE1D_OK;
    const int64_t grid = (int64_t)occ * p->sms;
    const int64_t B = p->B, nrows = P.L1 / 2 + 1;
    const int64_t tiles = (p->ns.M + kInterpTile - 1) / kInterpTile + (p->nr.M + kInterpTile - 1) / kInterpTile;
    const int64_t units = std::max({p->ns.nunits, B * P.L2, B * nrows, tiles});
    if (grid < 2) return WAVE1D_OK;
    int rc = balloc(p, &p->bar, (size_t)kBNumCounters);
    if (rc) return rc;
    if (cudaMemsetAsync(p->bar, 0, kBNumCounters * sizeof(unsigned), p->s) != cudaSuccess)
        return bfail(WAVE1D_ECUDA, "counter initialisation");
    p->W = w;
    p->pgrid = (unsigned)grid;
    p->psmem = sm;
    p->H = (int)std::max<int64_t>(1, std::min<int64_t>(units, grid / 2));
    p->persist = true;
    return WAVE1D_OK;
}

int launch_batch_step(wave1d_batch_t p, double* sig_hist) {
    BatchStep a;
    a.g = p->g;
    a.g.sig_hist = sig_hist;
    a.views = p->d_views;
    a.B = p->B;
    a.H = p->H;
    a.ns = p->ns;
    a.nr = p->nr;
    a.perm_s = p->perm_s;
    a.perm_r = p->perm_r;
    a.inst_of = p->inst_of;
    a.pulse = p->pulse;
    a.c = p->c;
    a.u = p->u;
    a.ur = p->ur;
    a.bar = p->bar;
    void* args[] = {&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->pgrid);
    cfg.blockDim = dim3(kBStepThreads);
    cfg.dynamicSmemBytes = p->psmem;
    cfg.stream = p->s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BCK(cudaLaunchKernelExC(&cfg, batch_step_kernel(p->W), args));
    return WAVE1D_OK;
}

// queue one step of every instance
int enqueue_batch_step(wave1d_batch_t p, double* sig_hist) {
    if (p->persist) return launch_batch_step(p, sig_hist);
    const Params& P = p->bt.g.P;
    DevPlan d = p->g;
    d.sig_hist = sig_hist;
    cudaStream_t s = p->s;
    const int T = 256;
    auto blocks = [](int64_t work, int per) { return (unsigned)std::max<int64_t>(1, (work + per - 1) / per); };
    const unsigned B = (unsigned)p->B;
    const int64_t items = d.l_nitems + d.r_nitems;
    k_local_items<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, (int64_t)p->sms * 4)), T, 0, s>>>(d);
    // history part: batched FP64 spreading, per-instance FFT columns, FIR tails, rows + modes,
    // inverse columns, batched interpolation
    k_mx_gather<<<blocks(P.M, T), T, 0, s>>>(d, p->perm_s, p->c);
    int rc = wave1d_nufft_spread(p->nu_s, p->c, p->grids);
    if (rc) return bfail(rc, std::string("batched spreading: ") + wave1d_nufft_strerror());
    const int l1 = 31 - __builtin_clz((unsigned)P.L1);
    const int t1 = std::max(32, std::min(P.L1 / 2, 512));
    k_bfft_cols<<<dim3(P.L2, B), t1, fft_smem_bytes(P.L1), s>>>((const double2*)p->grids, (double2*)p->work,
                                                                (const double2*)d.twiddle, P.L, P.L1, P.L2, l1);
    k_bhist_tail<<<dim3((P.K + 1 + kTailModes - 1) / kTailModes, B), 8 * kTailModes, 0, s>>>(p->d_views);
    k_bhist_rows<<<dim3(P.L1 / 2 + 1, B), T, rows_phase_smem(P.L2), s>>>(p->d_views);
    const unsigned tc = (unsigned)std::max(32, std::min(P.L1, 1024));
    k_bhist_icols<<<dim3(P.L2, B), tc, icols_phase_smem(P.L1), s>>>(p->d_views);
    rc = wave1d_nufft_interp(p->nu_s, p->grids, p->u);
    if (rc) return bfail(rc, std::string("batched interpolation: ") + wave1d_nufft_strerror());
    k_b_rhs<<<blocks(P.M, T), T, 0, s>>>(d, p->perm_s, p->u, p->inst_of, p->pulse);
    if (P.R > 0) {
        rc = wave1d_nufft_interp(p->nu_r, p->grids, p->ur);
        if (rc) return bfail(rc, std::string("batched interpolation: ") + wave1d_nufft_strerror());
        k_mx_receivers<<<blocks(P.R, T), T, 0, s>>>(P.R, p->perm_r, p->ur, d.uHr);
    }
    k_solve<<<blocks((d.n_sgroups + d.n_big) * 32, T), T, 0, s>>>(d);
    BCK(cudaGetLastError());
    return WAVE1D_OK;
}

// the joined instances on the device: tables, per-instance views, pulses, the batched NUFFT plans of
// the springs and of the receivers, and the one-launch step
int upload_joined_part(wave1d_batch_t p, const std::vector<int>& joined, const double* pulse, double tol,
                       const wave1d_opts& o) {
    const Params& P = p->bt.g.P;
    int rc;
    if ((rc = upload_joined(p)) || (rc = upload_views(p))) return rc;
    std::vector<double> pl((size_t)3 * p->B);
    for (int k = 0; k < p->B; k++) {
        const int b = joined[k];
        pl[3 * k] = pulse[3 * b];
        pl[3 * k + 1] = pulse[3 * b + 1];
        pl[3 * k + 2] = 1.0 / pulse[3 * b + 2];
    }
    if ((rc = bupload(p, pl, &p->pulse)) || (rc = bupload(p, p->bt.inst_of, &p->inst_of))) return rc;
    if ((rc = balloc(p, &p->c, (size_t)P.M)) || (rc = balloc(p, &p->u, (size_t)P.M))) return rc;
    // batched NUFFT plans of the springs and of the receivers: the instances' fine grids, kernel
    // (width from tol, as each instance's plan) and deconvolution
    rc = wave1d_nufft_plan_many(p->bt.g.x.data(), p->bt.moff.data(), p->B, P.K, tol, 0, (void*)p->s, &p->nu_s);
    if (rc) return bfail(rc, std::string("batched NUFFT plan: ") + wave1d_nufft_strerror());
    std::vector<int64_t> perm((size_t)P.M);
    if ((rc = wave1d_nufft_perm(p->nu_s, perm.data()))) return bfail(rc, wave1d_nufft_strerror());
    if ((rc = bupload(p, perm, &p->perm_s))) return rc;
    if (P.R > 0) {
        rc = wave1d_nufft_plan_many(p->bt.g.xr.data(), p->bt.roff.data(), p->B, P.K, tol, 0, (void*)p->s, &p->nu_r);
        if (rc) return bfail(rc, std::string("batched NUFFT plan of the receivers: ") + wave1d_nufft_strerror());
        std::vector<int64_t> permr((size_t)P.R);
        if ((rc = wave1d_nufft_perm(p->nu_r, permr.data()))) return bfail(rc, wave1d_nufft_strerror());
        if ((rc = bupload(p, permr, &p->perm_r)) || (rc = balloc(p, &p->ur, (size_t)P.R))) return rc;
    }
    if (cudaFuncSetAttribute(k_bhist_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_phase_smem(P.L2)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_bfft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem_bytes(P.L1)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_bhist_icols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)icols_phase_smem(P.L1)) !=
            cudaSuccess)
        return bfail(WAVE1D_ECUDA, "cannot size the shared memory of the history passes");
    p->g.spin_limit = o.spin_limit > 0 ? (unsigned)o.spin_limit : (1u << 22);
    return setup_batch_step(p, o);
}

// queue one step of every instance: the joined instances (one launch or one launch per pass), then
// each instance without pair lists as a branch of its own, concurrent with the others
int enqueue_all(wave1d_batch_t p, bool with_sigma) {
    int rc;
    if (p->has_joined && (rc = enqueue_batch_step(p, with_sigma ? p->sig_hist : nullptr))) return rc;
    if (p->sub.empty()) return WAVE1D_OK;
    BCK(cudaEventRecord(p->ev_fork, p->s));
    for (size_t i = 0; i < p->sub.size(); i++)
        if ((rc = plan_branch_step(p->sub[i], p->ev_fork, with_sigma ? p->sub_sig[i] : nullptr)))
            return bfail(rc, std::string("instance plan: ") + wave1d_strerror(rc));
    for (wave1d_plan_t q : p->sub)
        if ((rc = plan_branch_join(q, p->s))) return bfail(rc, std::string("instance plan: ") + wave1d_strerror(rc));
    return WAVE1D_OK;
}

// rows [row0, row0 + rows) of the rings (ring row slot0 ..) into rows first .. of the outputs
int copy_rows(wave1d_batch_t p, double* u_rec, double* sigma, cudaMemcpyKind kind, int64_t slot0, int64_t first,
              int64_t rows) {
    const size_t d = sizeof(double);
    if (p->has_joined) {
        const Params& P = p->bt.g.P;
        for (size_t i = 0; u_rec && i < p->seg_r.size(); i += 3)
            BCK(cudaMemcpy2DAsync(u_rec + first * p->R_all + p->seg_r[i + 1], p->R_all * d,
                                  p->g.rec_hist + slot0 * P.R + p->seg_r[i], P.R * d, p->seg_r[i + 2] * d, rows, kind, p->s));
        for (size_t i = 0; sigma && i < p->seg_m.size(); i += 3)
            BCK(cudaMemcpy2DAsync(sigma + first * p->M_all + p->seg_m[i + 1], p->M_all * d,
                                  p->sig_hist + slot0 * P.M + p->seg_m[i], P.M * d, p->seg_m[i + 2] * d, rows, kind, p->s));
    }
    for (size_t k = 0; k < p->sub.size(); k++) {
        const PlanHooks& h = p->sub_hooks[k];
        if (u_rec && h.R > 0)
            BCK(cudaMemcpy2DAsync(u_rec + first * p->R_all + p->sub_roff[k], p->R_all * d, h.rec_hist + slot0 * h.R,
                                  h.R * d, h.R * d, rows, kind, p->s));
        if (sigma)
            BCK(cudaMemcpy2DAsync(sigma + first * p->M_all + p->sub_moff[k], p->M_all * d, p->sub_sig[k] + slot0 * h.M,
                                  h.M * d, h.M * d, rows, kind, p->s));
    }
    return WAVE1D_OK;
}

}  // namespace

extern "C" {

int wave1d_batch_plan(int n_inst, const int64_t* offsets, const double* x, const double* beta, const double* pulse,
                      const int64_t* r_offsets, const double* xr, double dt, int64_t Nt, double tol,
                      const wave1d_opts* opts, wave1d_batch_t* out) {
    if (!out) return bfail(WAVE1D_EINVAL, "out is NULL");
    *out = nullptr;
    g_batch_error.clear();
    if (n_inst < 1 || !offsets || !x || !beta || !pulse) return bfail(WAVE1D_EINVAL, "need instances, x, beta and pulses");
    if (offsets[0] != 0) return bfail(WAVE1D_EINVAL, "offsets[0] must be 0");
    for (int b = 0; b < n_inst; b++) {
        if (offsets[b + 1] <= offsets[b]) return bfail(WAVE1D_EINVAL, "every instance needs a spring");
        if (r_offsets && r_offsets[b + 1] <= r_offsets[b]) return bfail(WAVE1D_EINVAL, "every instance needs a receiver");
        if (!(pulse[3 * b + 2] > 0.0) || !std::isfinite(pulse[3 * b]) || !std::isfinite(pulse[3 * b + 1]))
            return bfail(WAVE1D_EINVAL, "pulse widths must be positive and parameters finite");
    }
    if (r_offsets && (r_offsets[0] != 0 || !xr)) return bfail(WAVE1D_EINVAL, "bad receivers");
    if (!(dt > 0.0) || Nt < 1 || !(tol > 0.0 && tol < 0.1)) return bfail(WAVE1D_EINVAL, "need dt > 0, Nt >= 1, 0 < tol < 0.1");
    wave1d_opts o;
    if (opts) o = *opts;
    else wave1d_opts_default(&o);
    if (o.p < 2 || o.p > 16 || (o.p % 2) != 0) return bfail(WAVE1D_EINVAL, "p must be even, 2..16");
    if (o.precision != 0 || o.nufft_w != 0)
        return bfail(WAVE1D_EINVAL, "the batched march runs in FP64 with the kernel width of its tolerance");
    if (o.local_weights < 0 || o.local_weights > 2)
        return bfail(WAVE1D_EINVAL, "local_weights of a batched plan: 0 stored, 1 none, 2 chosen per instance");
    if (o.max_block <= 0) o.max_block = 4096;
    if (o.max_local_bytes <= 0) o.max_local_bytes = (int64_t)16 << 30;

    wave1d_batch_t p = new (std::nothrow) wave1d_batch_s();
    if (!p) return bfail(WAVE1D_ENOMEM, "host allocation");
    auto cleanup = [&](int code) {
        wave1d_batch_destroy(p);
        return code;
    };
    p->n_inst = n_inst;
    p->M_all = offsets[n_inst];
    p->R_all = r_offsets ? r_offsets[n_inst] : 0;
    p->Nt = Nt;
    auto R_of = [&](int b) { return r_offsets ? r_offsets[b + 1] - r_offsets[b] : (int64_t)0; };
    // the form of each instance and the joined ones' own tables (batch_host.cpp), then joined
    std::vector<HostPlan> inst;
    std::vector<int> joined;
    std::string err;
    if (int rc = batch_instances(n_inst, offsets, x, beta, r_offsets, xr, dt, Nt, tol, o, p->form, joined, inst, err))
        return cleanup(bfail(rc, err));
    p->B = (int)joined.size();
    p->has_joined = p->B > 0;
    if (p->has_joined) {
        if (int rc = join_instances(inst, p->bt, err)) return cleanup(bfail(rc, err));
        // output columns of the joined rings, runs of consecutive instances merged
        for (int k = 0; k < p->B; k++) {
            const int b = joined[k];
            const int64_t add[2][3] = {{p->bt.moff[k], offsets[b], offsets[b + 1] - offsets[b]},
                                       {p->bt.roff[k], r_offsets ? r_offsets[b] : 0, R_of(b)}};
            for (int t = 0; t < 2; t++) {
                std::vector<int64_t>& seg = t ? p->seg_r : p->seg_m;
                if (add[t][2] == 0) continue;
                const size_t n = seg.size();
                if (n && seg[n - 3] + seg[n - 1] == add[t][0] && seg[n - 2] + seg[n - 1] == add[t][1]) seg[n - 1] += add[t][2];
                else seg.insert(seg.end(), add[t], add[t] + 3);
            }
        }
    }
    inst.clear();
    p->user = (cudaStream_t)o.stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) return cleanup(bfail(WAVE1D_ECUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(bfail(WAVE1D_ECUDA, "stream/event creation failed"));
    if (cudaEventRecord(p->ev_in, p->user) != cudaSuccess || cudaStreamWaitEvent(p->s, p->ev_in, 0) != cudaSuccess)
        return cleanup(bfail(WAVE1D_ECUDA, "stream ordering failed"));
    int rc;
    if (p->has_joined) {
        if ((rc = upload_joined_part(p, joined, pulse, tol, o))) return cleanup(rc);
    }
    // the instances without pair lists: one plan each
    wave1d_opts so = o;
    so.local_weights = 1;
    for (int b = 0; b < n_inst; b++) {
        if (p->form[b] != 1) continue;
        wave1d_plan_t q = nullptr;
        const std::string at = "instance " + std::to_string(b) + ": ";
        rc = wave1d_plan(x + offsets[b], beta + offsets[b], offsets[b + 1] - offsets[b], WAVE1D_PERIODIC, dt, Nt, tol, &so,
                         &q);
        if (rc) return cleanup(bfail(rc, at + wave1d_strerror(rc)));
        p->sub.push_back(q);
        if ((rc = wave1d_set_incident_gaussians(q, 1, pulse + 3 * b, pulse + 3 * b + 1, pulse + 3 * b + 2)) ||
            (R_of(b) > 0 && (rc = wave1d_set_receivers(q, xr + r_offsets[b], R_of(b)))))
            return cleanup(bfail(rc, at + wave1d_strerror(rc)));
        PlanHooks hk;
        if ((rc = plan_hooks(q, hk))) return cleanup(bfail(rc, at + wave1d_strerror(rc)));
        if (hk.chunk != p->chunk) return cleanup(bfail(WAVE1D_EINVAL, at + "ring length differs from the batch's"));
        p->sub_hooks.push_back(hk);
        p->sub_sig.push_back(nullptr);
        p->sub_moff.push_back(offsets[b]);
        p->sub_roff.push_back(r_offsets ? r_offsets[b] : 0);
    }
    if (cudaStreamSynchronize(p->s) != cudaSuccess) return cleanup(bfail(WAVE1D_ECUDA, "plan upload failed"));
    if (p->has_joined) {
        // the device holds the joined weights now: release the host copies
        std::vector<float>().swap(p->bt.g.litems.w);
        std::vector<float>().swap(p->bt.g.ritems.w);
        std::vector<double>().swap(p->bt.g.inv);
    }
    *out = p;
    return WAVE1D_OK;
}

int wave1d_batch_solve(wave1d_batch_t p, int64_t nsteps, double* u_rec, double* sigma, int out_on_device) {
    if (!p || nsteps < 0) return bfail(WAVE1D_EINVAL, "bad solve arguments");
    if (p->n + nsteps > p->Nt) return bfail(WAVE1D_EDONE, "nsteps beyond the Nt of the plan");
    BCK(cudaSetDevice(p->device));
    BCK(cudaEventRecord(p->ev_in, p->user));
    BCK(cudaStreamWaitEvent(p->s, p->ev_in, 0));
    if (sigma) {
        if (p->has_joined && !p->sig_hist) {
            int rc = balloc(p, &p->sig_hist, (size_t)p->chunk * p->bt.g.P.M);
            if (rc) return rc;
        }
        for (size_t k = 0; k < p->sub.size(); k++)
            if (!p->sub_sig[k]) {
                int rc = plan_sigma_ring(p->sub[k], &p->sub_sig[k]);
                if (rc) return bfail(rc, std::string("instance plan: ") + wave1d_strerror(rc));
            }
    }
    cudaGraphExec_t& ge = p->graph[sigma ? 1 : 0];
    if (!ge) {
        cudaGraph_t graph;
        BCK(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_all(p, sigma != nullptr);
        cudaError_t e = cudaStreamEndCapture(p->s, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return bfail(WAVE1D_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        BCK(cudaGraphInstantiate(&ge, graph, 0));
        BCK(cudaGraphDestroy(graph));
    }
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int64_t pending = 0;
    for (int64_t i = 0; i < nsteps; i++) {
        BCK(cudaGraphLaunch(ge, p->s));
        p->n++;
        pending++;
        if (p->n % p->chunk == 0 || i == nsteps - 1) {
            // rows (n - pending) mod chunk .. of the chunk buffers: contiguous, they never wrap
            const int64_t slot0 = (p->n - pending) % p->chunk, first = i + 1 - pending;
            int rc = copy_rows(p, p->R_all > 0 ? u_rec : nullptr, sigma, kind, slot0, first, pending);
            if (rc) return rc;
            pending = 0;
        }
    }
    for (wave1d_plan_t q : p->sub) plan_count_steps(q, nsteps);
    BCK(cudaEventRecord(p->ev_out, p->s));
    BCK(cudaStreamWaitEvent(p->user, p->ev_out, 0));
    // status words: the joined instances', then each plan's
    std::vector<int> st(1 + p->sub.size(), 0);
    if (p->has_joined) BCK(cudaMemcpyAsync(&st[0], p->g.status, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    for (size_t k = 0; k < p->sub.size(); k++)
        BCK(cudaMemcpyAsync(&st[k + 1], p->sub_hooks[k].status, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    BCK(cudaStreamSynchronize(p->s));
    for (int v : st) {
        if (v == WAVE1D_ETIMEOUT) return bfail(v, "a bounded wait between the blocks of the batched step kernel ran out");
        if (v == WAVE1D_ENOTCONV)
            return bfail(v, "the Jacobi sweeps of an instance without pair lists did not converge");
        if (v != 0) return bfail(v, "a density became non-finite during the march");
    }
    return WAVE1D_OK;
}

int wave1d_batch_step_kernel(wave1d_batch_t p) { return p ? (p->persist ? 1 : 0) : WAVE1D_EINVAL; }

int wave1d_batch_forms(wave1d_batch_t p, int* forms) {
    if (!p || !forms) return bfail(WAVE1D_EINVAL, "plan or forms is NULL");
    for (int b = 0; b < p->n_inst; b++) forms[b] = p->form[b];
    return WAVE1D_OK;
}

int wave1d_batch_destroy(wave1d_batch_t p) {
    if (!p) return WAVE1D_OK;
    if (p->s) cudaStreamSynchronize(p->s);
    for (auto& g : p->graph)
        if (g) cudaGraphExecDestroy(g);
    for (wave1d_plan_t q : p->sub) wave1d_destroy(q);
    if (p->nu_s) wave1d_nufft_destroy(p->nu_s);
    if (p->nu_r) wave1d_nufft_destroy(p->nu_r);
    for (void* a : p->allocs) cudaFree(a);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
    return WAVE1D_OK;
}

const char* wave1d_batch_strerror(void) { return g_batch_error.c_str(); }

}  // extern "C"
