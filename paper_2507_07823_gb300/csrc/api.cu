// C-ABI of the wave1d library (declared in include/wave1d.h).
//
// Each plan owns a private non-blocking stream.  Every call orders itself after the work already
// queued on the caller's stream (opts.stream, which may be the legacy default stream) and makes
// the caller's stream wait for the plan's work, so from the caller's point of view all work is
// stream-ordered on its own stream.  The private stream allows CUDA-graph capture of whole chunks
// of time steps (the legacy stream cannot be captured).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint_host.h"
#include "internal.h"
#include "plan_hooks.h"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {
__global__ void k_step(DevPlan P);
__global__ void k_hist_cols(DevPlan P, double2* Y);
__global__ void k_hist_rows(DevPlan P, const double2* Y, double2* T, int do_inverse);
__global__ void k_hist_icols(DevPlan P, const double2* T);
__global__ void k_hist_tail(DevPlan P);
__global__ void k_fft_cols(const double2*, double2*, const double2*, int, int, int, int, int);
__global__ void k_fft_rows(const double2*, double2*, const double2*, int, int, int, int, int);
__global__ void k_rbc_grid(DevPlan P);
__global__ void k_rbc_update(DevPlan P, int npts);
__global__ void k_interp(DevPlan P);
__global__ void k_local_items(DevPlan P);
__global__ void k_solve(DevPlan P);
__global__ void k_sigma_to_caller(DevPlan P, int64_t q, double* out);
__global__ void k_internal_to_caller(const int32_t* perm, int64_t M, const double* in, double* out);
__global__ void k_caller_to_internal(const int32_t* perm, int64_t M, const double* in, double* out);
__global__ void k_adj_receivers(int64_t M, int ring, int64_t n, const int64_t* ptr, const int32_t* rcv,
                                const int32_t* mrange, const int64_t* woff, const double* w, const double* ubar,
                                double* sb);
size_t adj_local_smem(int m_max, int warps);
__global__ void k_adj_take(int64_t M, double* slot_vals, double* out);
__global__ void k_adj_solve(DevPlan P, const int32_t* blk_of, const double* sigbar, const double* sigma_next,
                            const double* g_next, double* grad, double* gbar_next, double* cbar, double* uHbar);
__global__ void k_adj_local(DevPlan P, int64_t n, const double* cbar, double* sb);
__global__ void k_adj_gather(int64_t M, const int64_t* perm, const double* in, double* out);
__global__ void k_adj_scatter_add(int64_t M, const int64_t* perm, const double* in, double* acc);
__global__ void k_adj_modes_in(int K, const double* S1, const double* xr, const double* ubar, int64_t R, double* ab);
__global__ void k_adj_rbc_grid(int K, int npts, const int32_t* idx, const double* tw2K, const double* phi,
                               const double* dphi, const double* ab, const double* apb, double* uvbar);
__global__ void k_adj_rbc_update(int K, int npts, const int32_t* idx, const double* tw2K, const double* uvbar,
                                 double* ab, double* apb);
__global__ void k_adj_modes(int K, int W, int64_t n, const double* rot, const double* pq, double* ab, double* apb,
                            double* Sb, double* a2);
__global__ void k_ck_sig2(int64_t n, const double* sig, float2* sig2);
__global__ void k_ck_step(int64_t* step, int64_t n);
__global__ void k_mx_gather(DevPlan P, const int64_t* perm, double* c);
__global__ void k_mx_rhs(DevPlan P, const int64_t* perm, const double* u);
__global__ void k_mx_receivers(int64_t R, const int64_t* perm, const double* u, double* uHr);
__global__ void k_rs_local(DevPlan P, RangeDev R);
__global__ void k_rs_local_T(DevPlan P, RangeDev R, int64_t n, const double* cbar, double* sb);
__global__ void k_rs_adj_init(DevPlan P, RangeDev R, double* slot_vals, double* rhs);
__global__ void k_rs_adj_post(DevPlan P, RangeDev R, const double* sigma_next, const double* g_next, double* grad,
                              double* gbar_next, double* cbar, double* uHbar);
__global__ void k_rs_adj_receivers(DevPlan P, RangeDev R, int64_t n, const double* ubar, double* sb);
size_t rs_local_T_smem(int nint, int nm);
__global__ void k_rs_nearby_weights(DevPlan P, RangeDev R);
__global__ void k_rs_solve_init(DevPlan P, RangeDev R);
__global__ void k_rs_jacobi(DevPlan P, RangeDev R, int it);
__global__ void k_rs_store(DevPlan P, RangeDev R);
__global__ void k_rs_receivers(DevPlan P, RangeDev R);
__global__ void k_rs_finish(DevPlan P, RangeDev R);
__global__ void k_rs_count_terms(DevPlan P, RangeDev R, unsigned long long* total);
size_t rs_local_smem(int nint, int nm);
}  // namespace wave1d

using namespace wave1d;

namespace {
thread_local std::string g_last_error;

struct Graph {
    cudaGraphExec_t exec = nullptr;
    bool with_sigma = false;
};
}  // namespace

struct wave1d_plan_s {
    HostPlan hp;
    DevPlan dp{};
    cudaStream_t user = nullptr;      // caller's stream (may be the legacy default stream)
    cudaStream_t s = nullptr;         // private stream
    cudaStream_t s2 = nullptr;        // side stream for the local sum (joined within each step)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int sms = 1;                      // multiprocessors of the device
    int64_t n = 0;                    // host mirror of the device step counter
    std::vector<void*> allocs;
    int64_t bytes = 0;
    bool started = false;
    double* d_g = nullptr;            // internal-order forcing
    double* d_gstage = nullptr;       // caller-order staging for a host forcing vector
    double* d_pulse = nullptr;
    int chunk = 32;
    double* d_sig_hist = nullptr;
    Graph graphs[2];                  // chunk graphs without / with the sigma history
    Graph step_graphs[2];             // single-step graphs: ordinary step / projection step
    bool step_kernel = false;         // ordinary steps as one cooperative launch (k_step)
    unsigned step_grid = 0;           // its blocks (all resident) and dynamic shared memory
    size_t step_smem = 0;
    bool profiling = false;
    cudaEvent_t prof_ev[WAVE1D_NSTAGE + 1] = {};
    double prof_ms[WAVE1D_NSTAGE] = {};
    int64_t prof_steps = 0;
    // mixed precision (opts.precision = 1): FP32 NUFFT plans of the springs and of the receivers
    // (same fine grid and kernel as the plan's, width 7), their point orders and work arrays
    // sizes of the local-sum tables, kept for wave1d_get_info once the host copies of the weights
    // (FP64 CSR, m-ordered rows, work-item weights) are released after the upload
    int64_t info_pairs = 0, info_weights = 0, info_nearby = 0, info_local_bytes = 0;
    // no pair lists (opts.local_weights = 1): local sum over sorted index windows with the weights
    // from their polynomials in the distance, implicit part solved by Jacobi sweeps (range.cu)
    bool range = false;
    RangeDev rd{};
    size_t rs_smem = 0;
    int64_t info_range_pairs = 0;
    int64_t info_terms = 0;           // (pair, m) terms of the local sum per step
    bool mixed = false;
    wave1d_nufft_t nu_s = nullptr, nu_r = nullptr;
    int64_t *nu_perm_s = nullptr, *nu_perm_r = nullptr;
    double *nu_c = nullptr, *nu_u = nullptr, *nu_ur = nullptr;
};

namespace {

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(WAVE1D_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

template <typename T>
int dalloc(wave1d_plan_t p, T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) return fail(WAVE1D_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    p->allocs.push_back(ptr);
    p->bytes += (int64_t)(count * sizeof(T));
    *out = (T*)ptr;
    return WAVE1D_OK;
}

template <typename T>
int upload(wave1d_plan_t p, const std::vector<T>& v, T** out) {
    int rc = dalloc(p, out, v.size());
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p->s));
    return WAVE1D_OK;
}

template <typename T>
int zeros(wave1d_plan_t p, T** out, size_t count) {
    int rc = dalloc(p, out, count);
    if (rc) return rc;
    CK(cudaMemsetAsync(*out, 0, std::max<size_t>(count, 1) * sizeof(T), p->s));
    return WAVE1D_OK;
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// order the private stream after the caller's stream
int enter(wave1d_plan_t p) {
    CK(cudaSetDevice(p->device));
    CK(cudaEventRecord(p->ev_in, p->user));
    CK(cudaStreamWaitEvent(p->s, p->ev_in, 0));
    return WAVE1D_OK;
}

// order the caller's stream after the private stream
int leave(wave1d_plan_t p) {
    CK(cudaEventRecord(p->ev_out, p->s));
    CK(cudaStreamWaitEvent(p->user, p->ev_out, 0));
    return WAVE1D_OK;
}

struct ItemsDev {
    const int64_t* item_ptr;
    const int32_t* row;
    const int32_t* s0;
    const int32_t* len;
    const int64_t* wbase;
    const int32_t* src;
    const float* w;
};

int upload_items(wave1d_plan_t p, const LocalItems& L, ItemsDev& o) {
    int rc;
    int64_t* i64;
    int32_t* i32;
    float* f32;
    if ((rc = upload(p, L.item_ptr, &i64))) return rc;
    o.item_ptr = i64;
    if ((rc = upload(p, L.row, &i32))) return rc;
    o.row = i32;
    if ((rc = upload(p, L.s0, &i32))) return rc;
    o.s0 = i32;
    if ((rc = upload(p, L.len, &i32))) return rc;
    o.len = i32;
    if ((rc = upload(p, L.wbase, &i64))) return rc;
    o.wbase = i64;
    if ((rc = upload(p, L.src, &i32))) return rc;
    o.src = i32;
    if ((rc = upload(p, L.w, &f32))) return rc;
    o.w = f32;
    return WAVE1D_OK;
}

int upload_receivers(wave1d_plan_t p) {
    HostPlan& hp = p->hp;
    DevPlan& d = p->dp;
    d.R = hp.P.R;
    int rc = 0;
    int32_t* i32;
    double* f64;
    if ((rc = upload(p, hp.rc_i0, &i32))) return rc;
    d.rc_i0 = i32;
    if ((rc = upload(p, hp.rc_ker, &f64))) return rc;
    d.rc_ker = f64;
    if (p->range) {
        // receivers' local part over index windows: their positions, windows and chunk partials
        if ((rc = upload(p, hp.xr, &f64))) return rc;
        d.xr = f64;
        if ((rc = upload(p, hp.r_win, &i32))) return rc;
        p->rd.r_win = i32;
        int64_t most = 1;
        for (int64_t r = 0; r < d.R; r++) most = std::max<int64_t>(most, hp.r_win[2 * r + 1] - hp.r_win[2 * r]);
        p->rd.rchunks = (int)((most + 255) / 256);
        if ((rc = zeros(p, &p->rd.r_part, (size_t)p->rd.rchunks * std::max<int64_t>(1, d.R)))) return rc;
        if ((rc = zeros(p, &d.uHr, (size_t)std::max<int64_t>(1, d.R)))) return rc;
        if ((rc = zeros(p, &d.rec_hist, (size_t)p->chunk * std::max<int64_t>(1, d.R)))) return rc;
        d.r_nitems = 0;
        return WAVE1D_OK;
    }
    ItemsDev it;
    if ((rc = upload_items(p, hp.ritems, it))) return rc;
    d.r_mfirst = hp.ritems.m_first;
    d.r_nitems = (int64_t)hp.ritems.row.size();
    d.r_item_ptr = it.item_ptr;
    d.r_s0 = it.s0;
    d.r_len = it.len;
    d.r_wbase = it.wbase;
    d.r_src = it.src;
    d.r_w = it.w;
    if ((rc = zeros(p, &d.r_part, (size_t)std::max<int64_t>(1, d.r_nitems)))) return rc;
    // items of the local sum in decreasing length, so the last items taken are short ones
    {
        const int64_t NL = d.l_nitems, NR = d.r_nitems;
        std::vector<int32_t> order((size_t)(NL + NR));
        auto len = [&](int32_t o) { return o < NL ? hp.litems.len[o] : hp.ritems.len[o - NL]; };
        for (int64_t i = 0; i < NL + NR; i++) order[i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
        int32_t* ob;
        if ((rc = upload(p, order, &ob))) return rc;
        d.item_order = ob;
    }
    // m = 0 terms padded to a whole number of warps per receiver
    int64_t most = 0;
    for (int64_t r = 0; r < d.R; r++) most = std::max(most, hp.r0_ptr[r + 1] - hp.r0_ptr[r]);
    d.r0_stride = (int)((most + 31) / 32 * 32);
    std::vector<int32_t> psrc((size_t)d.R * d.r0_stride, 0);
    std::vector<double> pw((size_t)d.R * d.r0_stride, 0.0);
    for (int64_t r = 0; r < d.R; r++)
        for (int64_t e = hp.r0_ptr[r]; e < hp.r0_ptr[r + 1]; e++) {
            psrc[(size_t)r * d.r0_stride + (e - hp.r0_ptr[r])] = hp.r0_src[e];
            pw[(size_t)r * d.r0_stride + (e - hp.r0_ptr[r])] = hp.r0_w[e];
        }
    int32_t* i32b;
    if ((rc = upload(p, psrc, &i32b))) return rc;
    d.r0p_src = i32b;
    double* f64b;
    if ((rc = upload(p, pw, &f64b))) return rc;
    d.r0p_w = f64b;
    if ((rc = zeros(p, &d.uHr, (size_t)std::max<int64_t>(1, d.R)))) return rc;
    if ((rc = zeros(p, &d.rec_hist, (size_t)p->chunk * std::max<int64_t>(1, d.R)))) return rc;
    return WAVE1D_OK;
}

// items kernel: as many 8-warp blocks as are resident at once (four per SM); warps fetch items
// dynamically
unsigned local_grid(const wave1d_plan_t p) {
    const DevPlan& d = p->dp;
    int64_t items = d.l_nitems + d.r_nitems;
    int64_t want = (items + 7) / 8;
    int64_t cap = (int64_t)p->sms * 4;
    return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

bool is_rbc_step(const wave1d_plan_t p, int64_t n) {
    return p->hp.P.bc == WAVE1D_FREE && ((n + 1) % p->hp.P.rbc_period) == 0;
}

// queue one step n -> n+1 on the private stream; ev (optional) gets WAVE1D_NSTAGE + 1 events
// recorded between the stages
int enqueue_step(wave1d_plan_t p, int64_t n, const double* g_ext, double* sig_hist,
                 cudaEvent_t* ev = nullptr) {
    const Params& P = p->hp.P;
    DevPlan d = p->dp;
    d.g_ext = g_ext;
    d.sig_hist = sig_hist;
    cudaStream_t s = p->s;
    const int T = 256;
    auto blocks = [](int64_t work, int per) { return (unsigned)std::max<int64_t>(1, (work + per - 1) / per); };
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], s);
    };
    bool rbc = is_rbc_step(p, n);
    if (p->step_kernel && !rbc && !ev) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(p->step_grid);
        cfg.blockDim = dim3(kStepThreads);
        cfg.dynamicSmemBytes = p->step_smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, k_step, d));
        return WAVE1D_OK;
    }
    // The local sum needs only sigma^{<= n} and could overlap the history pipeline on the side
    // stream, but on GB300 the two slow each other down (the latency-bound history kernels wait
    // longer on an HBM the local sum keeps busy): measured 169 us per step concurrently against
    // 143 us back to back at M = 1e4, so they run back to back.
    bool fork = false;
    mark(WAVE1D_STAGE_LOCAL);
    if (fork) {
        cudaEventRecord(p->ev_fork, s);
        cudaStreamWaitEvent(p->s2, p->ev_fork, 0);
        k_local_items<<<local_grid(p), T, 0, p->s2>>>(d);
        cudaEventRecord(p->ev_join, p->s2);
    } else if (p->range) {
        k_rs_local<<<p->rd.nblk, kRsTargets, p->rs_smem, s>>>(d, p->rd);
    } else {
        k_local_items<<<local_grid(p), T, 0, s>>>(d);
    }
    // history pipeline: spreading + forward columns | forward rows + modes (+ inverse rows) |
    // [projection] | inverse columns
    double2* Y = (double2*)d.work;
    double2* Tb = (double2*)d.spec;
    const double2* tw = (const double2*)d.twiddle;
    int l1 = ilog2(P.L1), l2 = ilog2(P.L2);
    unsigned tc = (unsigned)std::max(32, std::min(P.L1, 1024));
    mark(WAVE1D_STAGE_SPREAD);
    if (p->mixed) {
        // FP32 spreading of sigma^n onto the fine grid, then the forward FFT's column pass
        int t1 = std::max(32, std::min(P.L1 / 2, 512));
        k_mx_gather<<<blocks(P.M, T), T, 0, s>>>(d, p->nu_perm_s, p->nu_c);
        int rc = wave1d_nufft_spread(p->nu_s, p->nu_c, d.grid);
        if (rc) return fail(rc, std::string("mixed spreading: ") + wave1d_nufft_strerror());
        k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), s>>>((const double2*)d.grid, Y, tw, P.L, P.L1, P.L2, l1, +1);
    } else {
        k_hist_cols<<<P.L2, 256, cols_phase_smem(P.L1), s>>>(d, Y);
    }
    mark(WAVE1D_STAGE_FFT_FWD);
    mark(WAVE1D_STAGE_MODES);
    k_hist_tail<<<(P.K + 1 + kTailModes - 1) / kTailModes, 8 * kTailModes, 0, s>>>(d);
    k_hist_rows<<<P.L1 / 2 + 1, T, rows_phase_smem(P.L2), s>>>(d, Y, Tb, rbc ? 0 : 1);
    mark(WAVE1D_STAGE_RBC);
    if (rbc) {
        int npts = (int)p->hp.rbc_idx.size();
        k_rbc_grid<<<npts, T, 0, s>>>(d);
        k_rbc_update<<<blocks(P.K + 1, 128), 128, 0, s>>>(d, npts);
    }
    mark(WAVE1D_STAGE_FFT_INV);
    if (rbc) {
        int t1 = std::max(32, std::min(P.L1 / 2, 512)), t2 = std::max(32, std::min(P.L2 / 2, 512));
        k_fft_cols<<<P.L2, t1, fft_smem_bytes(P.L1), s>>>((const double2*)d.spec2, (double2*)d.work, tw, P.L,
                                                          P.L1, P.L2, l1, -1);
        k_fft_rows<<<P.L1, t2, fft_smem_bytes(P.L2), s>>>((const double2*)d.work, (double2*)d.grid, tw, P.L,
                                                          P.L1, P.L2, l2, -1);
    } else {
        k_hist_icols<<<P.L2, tc, icols_phase_smem(P.L1), s>>>(d, Tb);
    }
    mark(WAVE1D_STAGE_INTERP);
    if (p->mixed) {
        // FP32 interpolation at the springs (then u_H and the right-hand side) and at the receivers
        int rc = wave1d_nufft_interp(p->nu_s, d.grid, p->nu_u);
        if (rc) return fail(rc, std::string("mixed interpolation: ") + wave1d_nufft_strerror());
        k_mx_rhs<<<blocks(P.M, T), T, 0, s>>>(d, p->nu_perm_s, p->nu_u);
        if (P.R > 0) {
            rc = wave1d_nufft_interp(p->nu_r, d.grid, p->nu_ur);
            if (rc) return fail(rc, std::string("mixed interpolation: ") + wave1d_nufft_strerror());
            k_mx_receivers<<<blocks(P.R, T), T, 0, s>>>(P.R, p->nu_perm_r, p->nu_ur, d.uHr);
        }
    } else {
        k_interp<<<blocks(P.M + P.R, kInterpPoints), 2 * kInterpPoints, 0, s>>>(d);
    }
    mark(WAVE1D_STAGE_SOLVE);
    if (fork) cudaStreamWaitEvent(s, p->ev_join, 0);
    if (p->range) {
        const unsigned rows = blocks(P.M, T), sweeps = (unsigned)std::min<int64_t>(blocks(P.M * 32, T), 16 * (int64_t)p->sms);
        k_rs_solve_init<<<rows, T, 0, s>>>(d, p->rd);
        for (int it = 1; it <= kRsMaxIter; it++) k_rs_jacobi<<<sweeps, T, 0, s>>>(d, p->rd, it);
        k_rs_store<<<rows, T, 0, s>>>(d, p->rd);
        mark(WAVE1D_STAGE_RECEIVERS);
        if (P.R > 0) k_rs_receivers<<<dim3((unsigned)p->rd.rchunks, (unsigned)P.R), T, 0, s>>>(d, p->rd);
        k_rs_finish<<<1, 32, 0, s>>>(d, p->rd);
        mark(WAVE1D_NSTAGE);
        CK(cudaGetLastError());
        return WAVE1D_OK;
    }
    k_solve<<<blocks((d.n_sgroups + d.n_big) * 32, T), T, 0, s>>>(d);
    mark(WAVE1D_STAGE_RECEIVERS);      // the receivers are read out by the solve's last block
    mark(WAVE1D_NSTAGE);
    CK(cudaGetLastError());
    return WAVE1D_OK;
}

int check_status(wave1d_plan_t p) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, p->dp.status, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    if (st == WAVE1D_ETIMEOUT) return fail(st, "a bounded wait between the blocks of the step kernel ran out");
    if (st == WAVE1D_ENOTCONV)
        return fail(st, "the Jacobi sweeps of the implicit solve did not converge (local_weights = 1)");
    if (st != 0) return fail(st, "a density became non-finite during the march");
    return WAVE1D_OK;
}

int build_graph(wave1d_plan_t p, Graph& g, bool with_sigma) {
    if (g.exec) return WAVE1D_OK;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
    // the chunk starts at a multiple of `chunk`, so step offsets inside it fix the projections
    int rc = WAVE1D_OK;
    for (int i = 0; i < p->chunk && rc == WAVE1D_OK; i++)
        rc = enqueue_step(p, i, nullptr, with_sigma ? p->d_sig_hist : nullptr);
    cudaError_t e = cudaStreamEndCapture(p->s, &graph);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(WAVE1D_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&g.exec, graph, 0));
    CK(cudaGraphDestroy(graph));
    g.with_sigma = with_sigma;
    return WAVE1D_OK;
}

// one step through the fastest path available: profiled eager, eager with external forcing or
// sigma history, else a replayed single-step graph
int run_step(wave1d_plan_t p, const double* g_ext, double* sig_hist) {
    int64_t n = p->n;
    if (p->profiling) {
        int rc = enqueue_step(p, n, g_ext, sig_hist, p->prof_ev);
        if (rc) return rc;
        CK(cudaEventSynchronize(p->prof_ev[WAVE1D_NSTAGE]));
        for (int i = 0; i < WAVE1D_NSTAGE; i++) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, p->prof_ev[i], p->prof_ev[i + 1]));
            p->prof_ms[i] += ms;
        }
        p->prof_steps++;
        return WAVE1D_OK;
    }
    if (g_ext || sig_hist) return enqueue_step(p, n, g_ext, sig_hist);
    Graph& g = p->step_graphs[is_rbc_step(p, n) ? 1 : 0];
    if (!g.exec) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_step(p, n, nullptr, nullptr);
        cudaError_t e = cudaStreamEndCapture(p->s, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(WAVE1D_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        CK(cudaGraphInstantiate(&g.exec, graph, 0));
        CK(cudaGraphDestroy(graph));
    }
    CK(cudaGraphLaunch(g.exec, p->s));
    return WAVE1D_OK;
}

void drop_graphs(wave1d_plan_t p) {
    for (auto& g : p->graphs)
        if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    for (auto& g : p->step_graphs)
        if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
}

}  // namespace

extern "C" {

int wave1d_opts_default(wave1d_opts* o) {
    if (!o) return fail(WAVE1D_EINVAL, "opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->p = 8;
    o->gamma = 0.5;
    o->Ng = 32;
    o->max_block = 4096;
    o->max_local_bytes = (int64_t)16 << 30;
    o->step_kernel = 1;
    return WAVE1D_OK;
}

const char* wave1d_strerror(int status) {
    if (!g_last_error.empty() && status != WAVE1D_OK) return g_last_error.c_str();
    switch (status) {
        case WAVE1D_OK: return "ok";
        case WAVE1D_EINVAL: return "invalid argument";
        case WAVE1D_EDOMAIN: return "input outside the method's domain";
        case WAVE1D_ENOMEM: return "out of memory";
        case WAVE1D_ECUDA: return "CUDA runtime error";
        case WAVE1D_ENONFINITE: return "non-finite density";
        case WAVE1D_EDONE: return "all planned steps taken";
        case WAVE1D_EUNSUPPORTED: return "size not supported by this build";
        case WAVE1D_ETIMEOUT: return "a bounded wait of the step kernel ran out";
        case WAVE1D_ENOTCONV: return "the iterative implicit solve did not converge";
        default: return "unknown status";
    }
}

int wave1d_plan(const double* x, const double* beta, int64_t M, int bc, double dt, int64_t Nt,
                double tol, const wave1d_opts* opts, wave1d_plan_t* out) {
    if (!out) return fail(WAVE1D_EINVAL, "out is NULL");
    *out = nullptr;
    g_last_error.clear();
    if (!x || !beta || M < 1 || M > INT32_MAX / 2) return fail(WAVE1D_EINVAL, "need x, beta and 1 <= M < 2^30");
    if (bc != WAVE1D_PERIODIC && bc != WAVE1D_FREE) return fail(WAVE1D_EINVAL, "bc must be WAVE1D_PERIODIC or WAVE1D_FREE");
    if (!(dt > 0.0) || Nt < 1 || !(tol > 0.0 && tol < 0.1)) return fail(WAVE1D_EINVAL, "need dt > 0, Nt >= 1, 0 < tol < 0.1");
    wave1d_opts o;
    if (opts) o = *opts;
    else wave1d_opts_default(&o);
    if (o.p < 2 || o.p > 16 || (o.p % 2) != 0) return fail(WAVE1D_EINVAL, "p must be even, 2..16");
    if (!(o.gamma > 0.0 && o.gamma < 1.0)) return fail(WAVE1D_EINVAL, "gamma must lie in (0, 1)");
    if (o.max_block <= 0) o.max_block = 4096;
    if (o.max_local_bytes <= 0) o.max_local_bytes = (int64_t)16 << 30;
    if (o.precision != 0 && o.precision != 1) return fail(WAVE1D_EINVAL, "precision must be 0 (FP64) or 1 (mixed)");
    if (o.local_weights != 0 && o.local_weights != 1)
        return fail(WAVE1D_EINVAL, "local_weights must be 0 (stored) or 1 (computed per pair)");
    if (o.local_weights == 1) o.step_kernel = 0;   // the range-mode step is its own sequence of launches
    if (o.precision == 1) {
        if (o.nufft_w != 0 && o.nufft_w != 7) return fail(WAVE1D_EINVAL, "mixed precision uses the width-7 NUFFT kernel");
        o.nufft_w = 7;          // the FP32 kernels' width: the plan's grid, kernel and deconvolution match them
        o.step_kernel = 0;      // the FP32 passes run as their own launches
    }

    wave1d_plan_t p = new (std::nothrow) wave1d_plan_s();
    if (!p) return fail(WAVE1D_ENOMEM, "host allocation");
    std::string err;
    int rc = build_host_plan(x, beta, M, bc, dt, Nt, tol, o.p, o.gamma, o.W, o.NL, o.Ng, o.nufft_w,
                             o.rbc_period, o.max_block, o.max_local_bytes, p->hp, err, o.local_weights == 1);
    if (rc == WAVE1D_OK && o.local_weights == 1 && p->hp.rt.iv_dt >= p->hp.rt.nint) {
        rc = WAVE1D_EINVAL;
        err = "local_weights = 1 needs a window of at least two steps (W >= 2)";
    }
    if (rc == WAVE1D_OK && o.local_weights == 1 && p->hp.rt.nint >= 32768) {
        rc = WAVE1D_EUNSUPPORTED;
        err = "local_weights = 1: more than 32767 distance intervals (tolerance too small for dt)";
    }
    if (rc == WAVE1D_OK) {
        double none = 0.0;
        rc = build_receivers(p->hp, &none, 0, err);
    }
    if (rc != WAVE1D_OK) {
        delete p;
        return fail(rc, err);
    }
    const Params& P = p->hp.P;
    p->chunk = P.bc == WAVE1D_FREE ? P.rbc_period : 32;
    p->range = o.local_weights == 1;
    p->user = (cudaStream_t)o.stream;
    auto cleanup = [&](int code) {
        wave1d_destroy(p);
        return code;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return cleanup(fail(WAVE1D_ECUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        return cleanup(fail(WAVE1D_ECUDA, "cannot read the multiprocessor count"));
    // the history pipeline (main stream) has the critical path: highest priority; the local sum
    // (side stream) fills the remaining capacity at the lowest priority
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (cudaStreamCreateWithPriority(&p->s, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaStreamCreateWithPriority(&p->s2, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(WAVE1D_ECUDA, "stream/event creation failed"));
    if ((rc = enter(p))) return cleanup(rc);
    if (cudaFuncSetAttribute(k_hist_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cols_phase_smem(P.L1)) != cudaSuccess)
        return cleanup(fail(WAVE1D_ECUDA, "cannot size the shared memory of the column pass"));
    // one-launch step kernel: as many blocks as are resident at once, the history group one block
    // per column / row pair
    if (o.step_kernel) {
        size_t sm = std::max({cols_phase_smem(P.L1), rows_phase_smem(P.L2), icols_phase_smem(P.L1),
                              (size_t)kSolveStage * sizeof(double) * (kStepThreads / 32)});
        int occ = 0;
        if (cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step, kStepThreads, sm) != cudaSuccess)
            return cleanup(fail(WAVE1D_ECUDA, "cannot configure the step kernel"));
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, p->device);
        int64_t grid = (int64_t)occ * p->sms;
        // one history block per column / row pair / interpolation chunk, at most half the blocks
        int64_t units = std::max<int64_t>(std::max(P.L2, P.L1 / 2 + 1),
                                          (P.M + kInterpPoints - 1) / kInterpPoints);
        if (coop && occ > 0) {
            p->step_kernel = true;
            p->step_grid = (unsigned)grid;
            p->step_smem = sm;
            p->dp.hist_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(units, grid / 2));
        }
    }

    HostPlan& hp = p->hp;
    DevPlan& d = p->dp;
    d.M = P.M;
    d.R = 0;
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
    d.npulse = 0;
    d.dt = P.dt;
    d.chunk = p->chunk;
    d.rbc_h = P.h_rbc;
    // polls of a counter before a wait of the step kernel gives up (each poll sleeps 0.1-1 us)
    d.spin_limit = o.spin_limit > 0 ? (unsigned)o.spin_limit : (1u << 22);
    d.hold_unit = o.hold_unit != 0;
    int32_t* i32;
    int64_t* i64;
    double* f64;
#define UP(vec, field, tmp)                      \
    if ((rc = upload(p, vec, &tmp))) return cleanup(rc); \
    d.field = tmp;
    if ((rc = zeros(p, &d.step, 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.item_ctr, 1))) return cleanup(rc);
    if ((rc = zeros(p, &d.status, 1))) return cleanup(rc);
    if ((rc = zeros(p, &d.bar, 16))) return cleanup(rc);
    if ((rc = zeros(p, &d.ftail, (size_t)4 * (P.K + 1)))) return cleanup(rc);
    if ((rc = zeros(p, &d.gforce, (size_t)P.M))) return cleanup(rc);
    UP(hp.x, x, f64);
    UP(hp.beta, beta, f64);
    UP(hp.perm, perm, i32);
    UP(hp.pq, pq, f64);
    UP(hp.rot, rot, f64);
    UP(hp.deconv1, deconv1, f64);
    UP(hp.deconv2, deconv2, f64);
    UP(hp.twiddle, twiddle, f64);
    UP(hp.modefac, modefac, f64);
    UP(hp.tw2K, tw2K, f64);
    UP(hp.g_ptr, g_ptr, i32);
    UP(hp.g_src, g_src, i32);
    UP(hp.g_w, g_w, f64);
    if ((rc = zeros(p, &d.Sring, (size_t)P.W * (P.K + 1) * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.alpha, (size_t)(P.K + 1) * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.alpha_p, (size_t)(P.K + 1) * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.grid, (size_t)P.nf))) return cleanup(rc);
    if ((rc = zeros(p, &d.spec, (size_t)P.L * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.spec2, (size_t)P.L * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.work, (size_t)P.L * 2))) return cleanup(rc);
    if ((rc = zeros(p, &d.rhs, (size_t)P.M))) return cleanup(rc);
    UP(hp.sp_i0, sp_i0, i32);
    UP(hp.sp_ker, sp_ker, f64);
    if ((rc = zeros(p, &d.uH, (size_t)P.M))) return cleanup(rc);
    if (p->range) {
        // the weights' polynomials, positions as float pairs, index windows, the implicit part's
        // weights (computed on the device below) and the solver's work arrays
        const RangeTables& rt = hp.rt;
        RangeDev& rd = p->rd;
        rd.nint = rt.nint;
        rd.nm = rt.nm;
        rd.iv_dt = rt.iv_dt;
        rd.nblk = (int)((P.M + kRsTargets - 1) / kRsTargets);
        rd.delta = P.delta;
        float* f32;
        int32_t* r32;
        int64_t* r64;
        double* r64f;
        std::vector<int32_t> mr(rt.mr.begin(), rt.mr.end()), mr0(rt.mr0.begin(), rt.mr0.end());
        if ((rc = upload(p, rt.bp2, &f32))) return cleanup(rc);
        rd.bp2 = f32;
        if ((rc = upload(p, rt.ih, &f32))) return cleanup(rc);
        rd.ih = f32;
        if ((rc = upload(p, rt.coef, &f32))) return cleanup(rc);
        rd.coef = f32;
        if ((rc = upload(p, mr, &r32))) return cleanup(rc);
        rd.mr = r32;
        if ((rc = upload(p, mr0, &r32))) return cleanup(rc);
        rd.mr0 = r32;
        if ((rc = upload(p, rt.bp, &r64f))) return cleanup(rc);
        rd.bp = r64f;
        if ((rc = upload(p, rt.mid, &r64f))) return cleanup(rc);
        rd.mid = r64f;
        if ((rc = upload(p, rt.cheb, &r64f))) return cleanup(rc);
        rd.cheb = r64f;
        if ((rc = upload(p, rt.cell, &r32))) return cleanup(rc);
        rd.cell = r32;
        rd.cell_scale = rt.cell_scale;
        if ((rc = upload(p, hp.blk_win, &r32))) return cleanup(rc);
        rd.blk_win = r32;
        if ((rc = upload(p, hp.nb_lo, &r32))) return cleanup(rc);
        rd.nb_lo = r32;
        if ((rc = upload(p, hp.nb_cnt, &r32))) return cleanup(rc);
        rd.nb_cnt = r32;
        if ((rc = upload(p, hp.nb_off, &r64))) return cleanup(rc);
        rd.nb_off = r64;
        if ((rc = dalloc(p, &rd.nb_w, 2 * (size_t)std::max<int64_t>(1, hp.nb_off[P.M])))) return cleanup(rc);
        if ((rc = dalloc(p, &rd.diag, (size_t)P.M))) return cleanup(rc);
        for (int i = 0; i < 2; i++) {
            if ((rc = zeros(p, &rd.it64[i], (size_t)P.M))) return cleanup(rc);
            if ((rc = zeros(p, &rd.it2[i], 2 * (size_t)P.M))) return cleanup(rc);
        }
        if ((rc = zeros(p, &rd.stats, 2 * (size_t)(kRsMaxIter + 1)))) return cleanup(rc);
        if ((rc = zeros(p, &rd.iters, 1))) return cleanup(rc);
        p->rs_smem = rs_local_smem(rt.nint, rt.nm);
        if (cudaFuncSetAttribute(k_rs_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->rs_smem) !=
            cudaSuccess)
            return cleanup(fail(WAVE1D_ECUDA, "cannot size the shared memory of the range-mode local sum"));
        p->info_range_pairs = hp.range_pairs;
    }
    {
        ItemsDev it;
        if ((rc = upload_items(p, hp.litems, it))) return cleanup(rc);
        d.l_mfirst = hp.litems.m_first;
        d.l_nitems = (int64_t)hp.litems.row.size();
        d.l_item_ptr = it.item_ptr;
        d.l_row = it.row;
        d.l_s0 = it.s0;
        d.l_len = it.len;
        d.l_wbase = it.wbase;
        d.l_src = it.src;
        d.l_w = it.w;
        if ((rc = zeros(p, &d.l_part, (size_t)std::max<int64_t>(1, d.l_nitems)))) return cleanup(rc);
    }
    if ((rc = zeros(p, &d.clocal, (size_t)P.M))) return cleanup(rc);
    if ((rc = zeros(p, &d.sig, (size_t)P.M * P.ring))) return cleanup(rc);
    if ((rc = zeros(p, &d.sig2, (size_t)P.M * P.ring * 4))) return cleanup(rc);
    UP(hp.blk_ptr, blk_ptr, i64);
    UP(hp.blk_members, blk_members, i32);
    UP(hp.blk_inv_off, blk_inv_off, i64);
    UP(hp.inv, inv, f64);
    d.nblocks = (int64_t)hp.blk_ptr.size() - 1;
    UP(hp.sg_j, sg_j, i32);
    UP(hp.sg_meta, sg_meta, i32);
    UP(hp.sg_smax, sg_smax, i32);
    UP(hp.sg_icnt, sg_icnt, i32);
    UP(hp.big_row0, big_row0, i32);
    UP(hp.sg_off, sg_off, i64);
    UP(hp.sg_ip, sg_ip, i64);
    UP(hp.big_blk, big_blk, i64);
    UP(hp.sg_beta, sg_beta, f64);
    d.n_sgroups = (int64_t)hp.sg_smax.size();
    d.n_big = (int64_t)hp.big_blk.size();
    d.inv_len = (int64_t)hp.inv.size();
    UP(hp.rbc_idx, rbc_idx, i32);
    UP(hp.rbc_x, rbc_x, f64);
    UP(hp.rbc_phi, rbc_phi, f64);
    UP(hp.rbc_dphi, rbc_dphi, f64);
    if ((rc = zeros(p, &d.rbc_uv, std::max<size_t>(4, hp.rbc_idx.size() * 4)))) return cleanup(rc);
    if ((rc = dalloc(p, &p->d_g, (size_t)P.M))) return cleanup(rc);
    if ((rc = dalloc(p, &p->d_gstage, (size_t)P.M))) return cleanup(rc);
    if ((rc = upload_receivers(p))) return cleanup(rc);
    d.pulse = nullptr;
    {
        // sizes for wave1d_get_info, then the host copies of the weights go (the device holds them;
        // the items' lengths stay, for ordering the receivers' items when receivers are set)
        const LocalItems& L = hp.litems;
        p->info_pairs = (int64_t)hp.loc.src.size();
        if (!p->range) p->info_terms = (int64_t)hp.loc.w.size();
        p->info_weights = (int64_t)hp.lrows.w.size() / 2;
        p->info_nearby = hp.loc.nearby;
        p->info_local_bytes = (int64_t)(L.w.size() * sizeof(float) + L.src.size() * sizeof(int32_t) +
                                        (L.s0.size() + L.len.size()) * sizeof(int32_t) +
                                        L.wbase.size() * sizeof(int64_t)) +
                              8 * (int64_t)L.row.size();
    }
    if (o.precision == 1) {
        p->mixed = true;
        // tol 1e-6 gives the width-7 kernel: the same nf, kernel shape and deconvolution as the plan's
        rc = wave1d_nufft_plan(hp.x.data(), P.M, P.K, 1e-6, 1, (void*)p->s, &p->nu_s);
        if (rc) return cleanup(fail(rc, std::string("mixed NUFFT plan of the springs: ") + wave1d_nufft_strerror()));
        std::vector<int64_t> perm(P.M);
        if ((rc = wave1d_nufft_perm(p->nu_s, perm.data()))) return cleanup(fail(rc, wave1d_nufft_strerror()));
        if ((rc = upload(p, perm, &p->nu_perm_s))) return cleanup(rc);
        if ((rc = dalloc(p, &p->nu_c, (size_t)P.M))) return cleanup(rc);
        if ((rc = dalloc(p, &p->nu_u, (size_t)P.M))) return cleanup(rc);
    }
#undef UP
    if (p->range) {
        // the implicit part's weights (beta_j / 2) Q_0(d_jl) of every spring's dt-window
        k_rs_nearby_weights<<<(unsigned)std::min<int64_t>((P.M + 7) / 8, 64 * (int64_t)p->sms), 256, 0, p->s>>>(d, p->rd);
        // the local sum's terms per step (reported by wave1d_get_info)
        unsigned long long* cnt;
        if ((rc = zeros(p, &cnt, 1))) return cleanup(rc);
        k_rs_count_terms<<<(unsigned)std::min<int64_t>((P.M + 255) / 256, 8 * (int64_t)p->sms), 256, 0, p->s>>>(d, p->rd, cnt);
        if (cudaGetLastError() != cudaSuccess) return cleanup(fail(WAVE1D_ECUDA, "nearby weights kernel"));
        unsigned long long terms = 0;
        if (cudaMemcpyAsync(&terms, cnt, sizeof(terms), cudaMemcpyDeviceToHost, p->s) != cudaSuccess ||
            cudaStreamSynchronize(p->s) != cudaSuccess)
            return cleanup(fail(WAVE1D_ECUDA, "counting the local sum's terms"));
        p->info_terms = (int64_t)terms;
    }
    if ((rc = leave(p))) return cleanup(rc);
    if (cudaStreamSynchronize(p->s) != cudaSuccess) return cleanup(fail(WAVE1D_ECUDA, "plan upload failed"));
    // the uploads have completed: release the host copies of the weights
    hp.loc = LocalCSR();
    hp.lrows = LocalRows();
    std::vector<float>().swap(hp.litems.w);
    *out = p;
    return WAVE1D_OK;
}

int wave1d_set_incident_gaussians(wave1d_plan_t p, int n, const double* amp, const double* center,
                                  const double* width) {
    if (!p || n < 0 || (n > 0 && (!amp || !center || !width))) return fail(WAVE1D_EINVAL, "bad incident-wave arguments");
    if (p->started) return fail(WAVE1D_EINVAL, "set the incident wave before stepping");
    std::vector<double> h(3 * (size_t)std::max(n, 1), 0.0);
    for (int i = 0; i < n; i++) {
        if (!(width[i] > 0.0) || !std::isfinite(amp[i]) || !std::isfinite(center[i]))
            return fail(WAVE1D_EINVAL, "pulse widths must be positive and parameters finite");
        h[3 * i] = amp[i];
        h[3 * i + 1] = center[i];
        h[3 * i + 2] = 1.0 / width[i];
    }
    int rc = enter(p);
    if (rc) return rc;
    double* dptr;
    if ((rc = upload(p, h, &dptr))) return rc;
    p->dp.pulse = dptr;
    p->dp.npulse = n;
    drop_graphs(p);
    return leave(p);
}

int wave1d_set_receivers(wave1d_plan_t p, const double* xr, int64_t R) {
    if (!p || R < 0 || (R > 0 && !xr)) return fail(WAVE1D_EINVAL, "bad receiver arguments");
    if (p->started) return fail(WAVE1D_EINVAL, "set receivers before stepping");
    std::string err;
    int rc = build_receivers(p->hp, xr, R, err);
    if (rc) return fail(rc, err);
    if ((rc = enter(p))) return rc;
    if ((rc = upload_receivers(p))) return rc;
    if (p->mixed && R > 0) {
        if (p->nu_r) {
            wave1d_nufft_destroy(p->nu_r);
            p->nu_r = nullptr;
        }
        rc = wave1d_nufft_plan(p->hp.xr.data(), R, p->hp.P.K, 1e-6, 1, (void*)p->s, &p->nu_r);
        if (rc) return fail(rc, std::string("mixed NUFFT plan of the receivers: ") + wave1d_nufft_strerror());
        std::vector<int64_t> perm(R);
        if ((rc = wave1d_nufft_perm(p->nu_r, perm.data()))) return fail(rc, wave1d_nufft_strerror());
        if ((rc = upload(p, perm, &p->nu_perm_r))) return rc;
        if ((rc = dalloc(p, &p->nu_ur, (size_t)R))) return rc;
    }
    drop_graphs(p);
    return leave(p);
}

int wave1d_step(wave1d_plan_t p, const double* g_next, int g_on_device) {
    if (!p) return fail(WAVE1D_EINVAL, "plan is NULL");
    if (p->n >= p->hp.P.Nt) return fail(WAVE1D_EDONE, "all planned steps taken");
    int rc = enter(p);
    if (rc) return rc;
    const double* gext = nullptr;
    if (g_next) {
        const double* src = g_next;
        if (!g_on_device) {
            CK(cudaMemcpyAsync(p->d_gstage, g_next, p->hp.P.M * sizeof(double), cudaMemcpyHostToDevice, p->s));
            src = p->d_gstage;
        }
        k_caller_to_internal<<<(unsigned)((p->hp.P.M + 255) / 256), 256, 0, p->s>>>(p->dp.perm, p->hp.P.M, src, p->d_g);
        gext = p->d_g;
    }
    p->started = true;
    if ((rc = run_step(p, gext, nullptr))) return rc;
    p->n++;
    return leave(p);
}

}  // extern "C"

namespace {
// nsteps steps of wave1d_solve, queued (the caller holds the plan's device)
int solve_steps(wave1d_plan_t p, int64_t nsteps, double* u_rec, double* sigma, int out_on_device) {
    const Params& P = p->hp.P;
    int rc;
    p->started = true;
    if (sigma && !p->d_sig_hist) {
        if ((rc = dalloc(p, &p->d_sig_hist, (size_t)p->chunk * P.M))) return rc;
    }
    cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int64_t done = 0;
    while (done < nsteps) {
        int64_t rem = nsteps - done;
        int64_t slot0 = p->n % p->chunk;
        int64_t cnt;
        if (slot0 == 0 && rem >= p->chunk && !p->profiling) {
            Graph& g = p->graphs[sigma ? 1 : 0];
            if ((rc = build_graph(p, g, sigma != nullptr))) return rc;
            CK(cudaGraphLaunch(g.exec, p->s));
            cnt = p->chunk;
        } else {
            if ((rc = run_step(p, nullptr, sigma ? p->d_sig_hist : nullptr))) return rc;
            cnt = 1;
        }
        if (u_rec && P.R > 0)
            CK(cudaMemcpyAsync(u_rec + done * P.R, p->dp.rec_hist + slot0 * P.R, cnt * P.R * sizeof(double),
                               kind, p->s));
        if (sigma)
            CK(cudaMemcpyAsync(sigma + done * P.M, p->d_sig_hist + slot0 * P.M, cnt * P.M * sizeof(double),
                               kind, p->s));
        p->n += cnt;
        done += cnt;
    }
    return WAVE1D_OK;
}
}  // namespace

extern "C" {

int wave1d_solve(wave1d_plan_t p, int64_t nsteps, double* u_rec, double* sigma, int out_on_device) {
    if (!p || nsteps < 0) return fail(WAVE1D_EINVAL, "bad solve arguments");
    if (p->n + nsteps > p->hp.P.Nt) return fail(WAVE1D_EDONE, "nsteps beyond the Nt of the plan");
    int rc = enter(p);
    if (rc) return rc;
    if ((rc = solve_steps(p, nsteps, u_rec, sigma, out_on_device))) return rc;
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

int wave1d_read_receivers(wave1d_plan_t p, double* u, int on_device) {
    if (!p || (!u && p->hp.P.R > 0)) return fail(WAVE1D_EINVAL, "bad arguments");
    if (p->hp.P.R == 0) return WAVE1D_OK;
    int rc = enter(p);
    if (rc) return rc;
    if (p->n == 0) {
        std::vector<double> z(p->hp.P.R, 0.0);
        if (on_device)
            CK(cudaMemcpyAsync(u, z.data(), z.size() * sizeof(double), cudaMemcpyHostToDevice, p->s));
        else
            std::memcpy(u, z.data(), z.size() * sizeof(double));
    } else {
        int64_t slot = (p->n - 1) % p->chunk;
        CK(cudaMemcpyAsync(u, p->dp.rec_hist + slot * p->hp.P.R, p->hp.P.R * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->s));
    }
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

int wave1d_get_sigma(wave1d_plan_t p, double* out, int on_device) {
    if (!p || !out) return fail(WAVE1D_EINVAL, "bad arguments");
    int rc = enter(p);
    if (rc) return rc;
    const Params& P = p->hp.P;
    double* dst = on_device ? out : p->d_gstage;
    k_sigma_to_caller<<<(unsigned)((P.M + 255) / 256), 256, 0, p->s>>>(p->dp, p->n, dst);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(out, p->d_gstage, P.M * sizeof(double), cudaMemcpyDeviceToHost, p->s));
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

// ---------------------------------------------------------------------------------------------
// checkpoint / resume: the state that evolves with the march (step counter, status word, density
// rings, mode coefficients and their S history, receiver history), behind a header that names
// the plan's sizes.  Everything else a step uses is either fixed by the plan or rebuilt each step.
// ---------------------------------------------------------------------------------------------
}  // extern "C"

namespace wave1d {

int plan_hooks(wave1d_plan_t p, PlanHooks& out) {
    if (!p) return fail(WAVE1D_EINVAL, "plan is NULL");
    out.M = p->hp.P.M;
    out.R = p->hp.P.R;
    out.Nt = p->hp.P.Nt;
    out.chunk = p->chunk;
    out.rec_hist = p->dp.rec_hist;
    out.status = p->dp.status;
    return WAVE1D_OK;
}

int plan_branch_step(wave1d_plan_t p, cudaEvent_t fork, double* sig_hist) {
    CK(cudaStreamWaitEvent(p->s, fork, 0));
    p->started = true;
    return enqueue_step(p, p->n, nullptr, sig_hist);
}

int plan_branch_join(wave1d_plan_t p, cudaStream_t s) {
    CK(cudaEventRecord(p->ev_join, p->s));
    CK(cudaStreamWaitEvent(s, p->ev_join, 0));
    return WAVE1D_OK;
}

int plan_sigma_ring(wave1d_plan_t p, double** out) {
    if (!p->d_sig_hist) {
        int rc = dalloc(p, &p->d_sig_hist, (size_t)p->chunk * p->hp.P.M);
        if (rc) return rc;
    }
    *out = p->d_sig_hist;
    return WAVE1D_OK;
}

void plan_count_steps(wave1d_plan_t p, int64_t k) { p->n += k; }

}  // namespace wave1d

namespace {

struct StateHeader {
    char magic[8];
    uint32_t version, reserved;
    int64_t M, R, K, W, ring, chunk, n;
    int32_t status, pad;
};

struct StatePart {
    void* dev;
    size_t bytes;
};

std::vector<StatePart> state_parts(wave1d_plan_t p) {
    const Params& P = p->hp.P;
    const DevPlan& d = p->dp;
    const size_t K1 = (size_t)P.K + 1;
    return {{d.sig, sizeof(double) * (size_t)P.ring * P.M},
            {d.sig2, sizeof(float) * 4 * (size_t)P.ring * P.M},
            {d.Sring, sizeof(double) * 2 * (size_t)P.W * K1},
            {d.alpha, sizeof(double) * 2 * K1},
            {d.alpha_p, sizeof(double) * 2 * K1},
            {d.rec_hist, sizeof(double) * (size_t)p->chunk * std::max<int64_t>(1, d.R)}};
}

void fill_header(wave1d_plan_t p, StateHeader& h) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "WAVE1DS", 8);
    h.version = 1;
    h.M = p->hp.P.M;
    h.R = p->dp.R;
    h.K = p->hp.P.K;
    h.W = p->hp.P.W;
    h.ring = p->hp.P.ring;
    h.chunk = p->chunk;
    h.n = p->n;
}

}  // namespace

extern "C" {

int wave1d_state_size(wave1d_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(WAVE1D_EINVAL, "bad arguments");
    size_t b = sizeof(StateHeader);
    for (const StatePart& s : state_parts(p)) b += s.bytes;
    *bytes = b;
    return WAVE1D_OK;
}

int wave1d_state_save(wave1d_plan_t p, void* buf, size_t bytes) {
    if (!p || !buf) return fail(WAVE1D_EINVAL, "bad arguments");
    size_t need = 0;
    wave1d_state_size(p, &need);
    if (bytes < need) return fail(WAVE1D_EINVAL, "state buffer smaller than wave1d_state_size");
    int rc = enter(p);
    if (rc) return rc;
    CK(cudaStreamSynchronize(p->s));
    StateHeader h;
    fill_header(p, h);
    CK(cudaMemcpy(&h.status, p->dp.status, sizeof(int), cudaMemcpyDeviceToHost));
    char* out = (char*)buf;
    std::memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    for (const StatePart& s : state_parts(p)) {
        CK(cudaMemcpy(out, s.dev, s.bytes, cudaMemcpyDeviceToHost));
        out += s.bytes;
    }
    return leave(p);
}

int wave1d_state_load(wave1d_plan_t p, const void* buf, size_t bytes) {
    if (!p || !buf) return fail(WAVE1D_EINVAL, "bad arguments");
    size_t need = 0;
    wave1d_state_size(p, &need);
    if (bytes < need) return fail(WAVE1D_EINVAL, "state buffer smaller than wave1d_state_size");
    StateHeader h, mine;
    std::memcpy(&h, buf, sizeof(h));
    fill_header(p, mine);
    if (std::memcmp(h.magic, mine.magic, 8) != 0 || h.version != mine.version)
        return fail(WAVE1D_EINVAL, "not a wave1d state buffer of this version");
    if (h.M != mine.M || h.R != mine.R || h.K != mine.K || h.W != mine.W || h.ring != mine.ring ||
        h.chunk != mine.chunk)
        return fail(WAVE1D_EINVAL, "state was saved from a plan of other sizes");
    if (h.n < 0 || h.n > p->hp.P.Nt) return fail(WAVE1D_EINVAL, "saved step beyond the Nt of this plan");
    int rc = enter(p);
    if (rc) return rc;
    CK(cudaStreamSynchronize(p->s));
    const char* in = (const char*)buf + sizeof(h);
    for (const StatePart& s : state_parts(p)) {
        CK(cudaMemcpy(s.dev, in, s.bytes, cudaMemcpyHostToDevice));
        in += s.bytes;
    }
    int64_t step[2] = {h.n, 0};
    CK(cudaMemcpy(p->dp.step, step, sizeof(step), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->dp.status, &h.status, sizeof(int), cudaMemcpyHostToDevice));
    p->n = h.n;
    p->started = true;
    return leave(p);
}

int wave1d_sync(wave1d_plan_t p) {
    if (!p) return fail(WAVE1D_EINVAL, "plan is NULL");
    int rc = enter(p);
    if (rc) return rc;
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

int wave1d_get_info(wave1d_plan_t p, wave1d_info* info) {
    if (!p || !info) return fail(WAVE1D_EINVAL, "bad arguments");
    const Params& P = p->hp.P;
    std::memset(info, 0, sizeof(*info));
    info->M = P.M;
    info->R = P.R;
    info->Nt = P.Nt;
    info->n = p->n;
    info->K = P.K;
    info->NF = 2 * P.K + 1;
    info->W = P.W;
    info->m_max = P.m_max;
    info->p = P.p;
    info->NL = P.NL;
    info->Ng = P.Ng;
    info->nufft_w = P.nufft_w;
    info->nf = P.nf;
    info->rbc_period = P.rbc_period;
    info->dt = P.dt;
    info->tol = P.tol;
    info->b = P.b;
    info->delta = P.delta;
    info->local_pairs = p->range ? p->info_range_pairs : p->info_pairs;
    info->local_weights = p->info_weights;
    info->nearby_pairs = p->range ? p->hp.nb_off[p->hp.P.M] : p->info_nearby;
    info->blocks = (int64_t)p->hp.blk_ptr.size() - 1;
    info->max_block = p->hp.max_block;
    info->device_bytes = p->bytes;
    info->local_bytes = p->info_local_bytes;
    info->local_terms = p->info_terms;
    info->solve_sweeps = 0;
    if (p->range && p->n > 0) {
        int it = 0;
        if (cudaStreamSynchronize(p->s) != cudaSuccess ||
            cudaMemcpy(&it, p->rd.iters, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(WAVE1D_ECUDA, "reading the solve's sweep count");
        info->solve_sweeps = it;
    }
    return WAVE1D_OK;
}

int wave1d_inspect(wave1d_plan_t p, int array, double* host_out, int64_t count) {
    if (!p || !host_out) return fail(WAVE1D_EINVAL, "bad arguments");
    const Params& P = p->hp.P;
    int64_t need = 0;
    switch (array) {
        case WAVE1D_ARR_ALPHA:
        case WAVE1D_ARR_ALPHA_P:
        case WAVE1D_ARR_S_LAST: need = 2 * (int64_t)(P.K + 1); break;
        case WAVE1D_ARR_UH:
        case WAVE1D_ARR_LOCAL:
        case WAVE1D_ARR_PERM: need = P.M; break;
        case WAVE1D_ARR_SIGMA_RING: need = (int64_t)(P.m_max + 1) * P.M; break;
        default: return fail(WAVE1D_EINVAL, "unknown array");
    }
    if (count != need) return fail(WAVE1D_EINVAL, "count does not match the array size");
    int rc = enter(p);
    if (rc) return rc;
    CK(cudaStreamSynchronize(p->s));
    switch (array) {
        case WAVE1D_ARR_ALPHA:
            CK(cudaMemcpy(host_out, p->dp.alpha, need * sizeof(double), cudaMemcpyDeviceToHost));
            break;
        case WAVE1D_ARR_ALPHA_P:
            CK(cudaMemcpy(host_out, p->dp.alpha_p, need * sizeof(double), cudaMemcpyDeviceToHost));
            break;
        case WAVE1D_ARR_S_LAST: {
            if (p->n == 0) { std::fill(host_out, host_out + need, 0.0); break; }
            int slot = (int)((p->n - 1) % P.W);
            CK(cudaMemcpy(host_out, p->dp.Sring + (size_t)slot * need, need * sizeof(double), cudaMemcpyDeviceToHost));
            break;
        }
        case WAVE1D_ARR_UH:
        case WAVE1D_ARR_LOCAL: {
            k_internal_to_caller<<<(unsigned)((P.M + 255) / 256), 256, 0, p->s>>>(
                p->dp.perm, P.M, array == WAVE1D_ARR_UH ? p->dp.uH : p->dp.clocal, p->d_gstage);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(host_out, p->d_gstage, P.M * sizeof(double), cudaMemcpyDeviceToHost, p->s));
            CK(cudaStreamSynchronize(p->s));
            break;
        }
        case WAVE1D_ARR_SIGMA_RING:
            for (int m = 0; m <= P.m_max; m++) {
                k_sigma_to_caller<<<(unsigned)((P.M + 255) / 256), 256, 0, p->s>>>(p->dp, p->n - m, p->d_gstage);
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(host_out + (size_t)m * P.M, p->d_gstage, P.M * sizeof(double),
                                   cudaMemcpyDeviceToHost, p->s));
            }
            CK(cudaStreamSynchronize(p->s));
            break;
        case WAVE1D_ARR_PERM:
            for (int64_t j = 0; j < P.M; j++) host_out[j] = (double)p->hp.perm[j];
            break;
    }
    return leave(p);
}

int wave1d_profile(wave1d_plan_t p, int enable) {
    if (!p) return fail(WAVE1D_EINVAL, "plan is NULL");
    if (enable) {
        for (int i = 0; i <= WAVE1D_NSTAGE; i++)
            if (!p->prof_ev[i]) CK(cudaEventCreate(&p->prof_ev[i]));
        for (int i = 0; i < WAVE1D_NSTAGE; i++) p->prof_ms[i] = 0.0;
        p->prof_steps = 0;
    }
    p->profiling = enable != 0;
    return WAVE1D_OK;
}

int wave1d_profile_read(wave1d_plan_t p, double* ms, int nstage, int64_t* steps) {
    if (!p || !ms || nstage != WAVE1D_NSTAGE) return fail(WAVE1D_EINVAL, "bad arguments");
    CK(cudaStreamSynchronize(p->s));
    for (int i = 0; i < WAVE1D_NSTAGE; i++) ms[i] = p->prof_ms[i];
    if (steps) *steps = p->prof_steps;
    return WAVE1D_OK;
}

}  // extern "C"

namespace {
// work arrays of one adjoint call, released (after the stream drains) when the call returns
struct AdjointWork {
    cudaStream_t s = nullptr;
    std::vector<void*> ptrs;
    wave1d_nufft_t nu = nullptr;
    ~AdjointWork() {
        if (s) cudaStreamSynchronize(s);
        for (void* q : ptrs) cudaFree(q);
        if (nu) wave1d_nufft_destroy(nu);
    }
    template <typename T>
    int zeros(T** out, size_t count) {
        void* q = nullptr;
        count = std::max<size_t>(count, 1);
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return fail(WAVE1D_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        ptrs.push_back(q);
        *out = (T*)q;
        CK(cudaMemsetAsync(q, 0, count * sizeof(T), s));
        return WAVE1D_OK;
    }
    template <typename T>
    int upload(const std::vector<T>& v, T** out) {
        int rc = zeros(out, v.size());
        if (rc || v.empty()) return rc;
        CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return WAVE1D_OK;
    }
};

unsigned blocks_for(int64_t threads, int per_block, int64_t cap) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + per_block - 1) / per_block, cap));
}
}  // namespace

extern "C" {

}  // extern "C"

namespace {
// The reverse march of one call: its work arrays and tables (allocated by init, released with wk)
// and the transposed steps.  The adjoint state (sb, Sb, ab, apb) carries from one call of steps()
// to the next, so the reverse march can be taken in segments.
struct Reverse {
    AdjointWork wk;
    wave1d_plan_t p = nullptr;
    double *sb, *Sb, *ab, *apb, *a2, *S1, *tmp, *cbar, *uHbar, *gsum, *cnu, *unu, *xr, *uvbar, *rw;
    int32_t *dblk, *rrcv, *rmr;
    int64_t *dperm, *rptr, *rwoff;
    bool have_rcv = false;
    int npts = 0;
    size_t lsmem = 0;
    double* rrhs = nullptr;   // plans without pair lists: the transposed solve's right-hand side
    size_t tsmem = 0;
    static constexpr int kLocalWarps = 4;     // the transposed local sum: one warp per spring row

    int init(wave1d_plan_t pl) {
        p = pl;
        wk.s = p->s;
        const HostPlan& hp = p->hp;
        const Params& P = hp.P;
        const int64_t M = P.M;
        const int K1 = P.K + 1;
        int rc;
        if ((rc = wave1d_nufft_plan(hp.x.data(), M, P.K, P.tol, 0, (void*)p->s, &wk.nu)))
            return fail(rc, std::string("NUFFT plan of the springs: ") + wave1d_nufft_strerror());
        std::vector<int64_t> nperm(M);
        if ((rc = wave1d_nufft_perm(wk.nu, nperm.data()))) return fail(rc, wave1d_nufft_strerror());
        std::vector<int32_t> blk_of(M);
        for (size_t b = 0; b + 1 < hp.blk_ptr.size(); b++)
            for (int64_t e = hp.blk_ptr[b]; e < hp.blk_ptr[b + 1]; e++) blk_of[e] = (int32_t)b;
        npts = (int)hp.rbc_idx.size();
        ReceiverColumns rcol;
        receiver_columns(hp.rloc, M, rcol);
        have_rcv = P.R > 0 && !rcol.rcv.empty();
        if ((rc = wk.zeros(&sb, (size_t)P.ring * M)) || (rc = wk.zeros(&Sb, (size_t)P.W * K1 * 2)) ||
            (rc = wk.zeros(&ab, 2 * (size_t)K1)) || (rc = wk.zeros(&apb, 2 * (size_t)K1)) ||
            (rc = wk.zeros(&a2, 2 * (size_t)K1)) || (rc = wk.zeros(&S1, 2 * (size_t)K1)) ||
            (rc = wk.zeros(&tmp, (size_t)M)) || (rc = wk.zeros(&cbar, (size_t)M)) || (rc = wk.zeros(&uHbar, (size_t)M)) ||
            (rc = wk.zeros(&gsum, (size_t)M)) || (rc = wk.zeros(&cnu, (size_t)M)) || (rc = wk.zeros(&unu, (size_t)M)) ||
            (rc = wk.zeros(&uvbar, 2 * (size_t)std::max(npts, 1))) || (rc = wk.upload(hp.xr, &xr)) ||
            (rc = wk.upload(blk_of, &dblk)) || (rc = wk.upload(nperm, &dperm)) ||
            (rc = wk.upload(rcol.src_ptr, &rptr)) || (rc = wk.upload(rcol.rcv, &rrcv)) ||
            (rc = wk.upload(rcol.mrange, &rmr)) || (rc = wk.upload(rcol.woff, &rwoff)) ||
            (rc = wk.upload(hp.rloc.w, &rw)))
            return rc;
        if (p->range) {
            if ((rc = wk.zeros(&rrhs, (size_t)M))) return rc;
            tsmem = rs_local_T_smem(p->rd.nint, p->rd.nm);
            if (tsmem > 227 * 1024) return fail(WAVE1D_EUNSUPPORTED, "window too long for the transposed local sum");
            CK(cudaFuncSetAttribute(k_rs_local_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
            return WAVE1D_OK;
        }
        lsmem = adj_local_smem(P.m_max, kLocalWarps);
        if (lsmem > 227 * 1024) return fail(WAVE1D_EUNSUPPORTED, "window too long for the adjoint's local-sum accumulators");
        if (lsmem > 48 * 1024)
            CK(cudaFuncSetAttribute(k_adj_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
        return WAVE1D_OK;
    }

    // transposed steps n = n_hi - 1 down to n_lo; sig_rows: the device row of sigma^{n+1} (caller
    // order) is sig_rows + (n - row0) M; g, ubar, grad_g: full nsteps-row arrays (or null)
    int steps(int64_t n_hi, int64_t n_lo, const double* sig_rows, int64_t row0, const double* g, const double* ubar,
              bool want_beta, double* grad_g) {
        const Params& P = p->hp.P;
        const int64_t M = P.M, R = P.R;
        const int K = P.K, K1 = P.K + 1, ring = P.ring;
        const DevPlan& d = p->dp;
        const int64_t cap = (int64_t)p->sms * 8;
        const unsigned gM = blocks_for(M, 256, cap), gK = blocks_for(K1, 256, INT32_MAX);
        cudaStream_t s = p->s;
        int rc;
        for (int64_t n = n_hi - 1; n >= n_lo; n--) {
            const double* ub = R > 0 ? ubar + n * R : nullptr;
            if (p->range) {
                // plan without pair lists: receivers, solve and local sum transposed on the
                // range tables; the solve is the forward Jacobi sweeps on beta-scaled data
                const RangeDev& rd = p->rd;
                if (R > 0) k_rs_adj_receivers<<<gM, 256, 0, s>>>(d, rd, n, ub, sb);
                k_rs_adj_init<<<gM, 256, 0, s>>>(d, rd, sb + (int64_t)((n + 1) % ring) * M, rrhs);
                DevPlan dj = d;
                dj.rhs = rrhs;
                const unsigned sweeps = (unsigned)std::min<int64_t>(blocks_for(M * 32, 256, INT32_MAX), 16 * (int64_t)p->sms);
                for (int it = 1; it <= kRsMaxIter; it++) k_rs_jacobi<<<sweeps, 256, 0, s>>>(dj, rd, it);
                k_rs_adj_post<<<gM, 256, 0, s>>>(d, rd, sig_rows + (n - row0) * M, g ? g + n * M : nullptr,
                                                 want_beta ? gsum : nullptr, grad_g ? grad_g + n * M : nullptr, cbar, uHbar);
                if (n == 0) break;
                k_rs_local_T<<<(unsigned)((M + kRsTTargets - 1) / kRsTTargets), kRsTTargets, tsmem, s>>>(d, rd, n, cbar, sb);
            } else {
                if (have_rcv) k_adj_receivers<<<gM, 256, 0, s>>>(M, ring, n, rptr, rrcv, rmr, rwoff, rw, ub, sb);
                k_adj_take<<<gM, 256, 0, s>>>(M, sb + (int64_t)(((n + 1) % ring)) * M, tmp);
                k_adj_solve<<<gM, 256, 0, s>>>(d, dblk, tmp, sig_rows + (n - row0) * M, g ? g + n * M : nullptr,
                                               want_beta ? gsum : nullptr, grad_g ? grad_g + n * M : nullptr, cbar, uHbar);
                if (n == 0) break;
                if (d.l_nitems > 0)
                    k_adj_local<<<blocks_for(M * 32, 32 * kLocalWarps, INT32_MAX), 32 * kLocalWarps, lsmem, s>>>(d, n, cbar, sb);
            }
            k_adj_gather<<<gM, 256, 0, s>>>(M, dperm, uHbar, cnu);
            if ((rc = wave1d_nufft_type1(wk.nu, cnu, S1))) return fail(rc, wave1d_nufft_strerror());
            k_adj_modes_in<<<gK, 256, 0, s>>>(K, S1, xr, ub, R, ab);
            if (P.bc == WAVE1D_FREE && (n + 1) % P.rbc_period == 0 && npts > 0) {
                k_adj_rbc_grid<<<blocks_for(npts, 64, INT32_MAX), 64, 0, s>>>(K, npts, d.rbc_idx, d.tw2K, d.rbc_phi,
                                                                             d.rbc_dphi, ab, apb, uvbar);
                k_adj_rbc_update<<<gK, 256, 0, s>>>(K, npts, d.rbc_idx, d.tw2K, uvbar, ab, apb);
            }
            k_adj_modes<<<gK, 256, 0, s>>>(K, P.W, n, d.rot, d.pq, ab, apb, Sb, a2);
            if ((rc = wave1d_nufft_type2(wk.nu, a2, unu))) return fail(rc, wave1d_nufft_strerror());
            k_adj_scatter_add<<<gM, 256, 0, s>>>(M, dperm, unu, sb + (int64_t)(n % ring) * M);
            CK(cudaGetLastError());
        }
        return WAVE1D_OK;
    }

    int finish(double* grad_beta) {
        if (grad_beta)
            k_internal_to_caller<<<blocks_for(p->hp.P.M, 256, (int64_t)p->sms * 8), 256, 0, p->s>>>(p->dp.perm, p->hp.P.M,
                                                                                                  gsum, grad_beta);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(p->s));
        return WAVE1D_OK;
    }
};

int adjoint_checks(wave1d_plan_t p, int64_t nsteps, const double* ubar, double* grad_beta, double* grad_g) {
    if (nsteps < 1 || (!grad_beta && !grad_g))
        return fail(WAVE1D_EINVAL, "need nsteps >= 1 and grad_beta or grad_g");
    const Params& P = p->hp.P;
    if (p->range)
        for (double b : p->hp.beta)
            if (!(b > 0.0))
                return fail(WAVE1D_EINVAL, "the transposed solve of a plan without pair lists needs every stiffness > 0");
    if (nsteps > P.Nt) return fail(WAVE1D_EINVAL, "nsteps beyond the Nt of the plan");
    if (P.R > 0 && !ubar) return fail(WAVE1D_EINVAL, "ubar is NULL");
    if (grad_beta)
        for (double b : p->hp.beta)
            if (!(b > 0.0))
                return fail(WAVE1D_EINVAL, "dL/dbeta needs every stiffness > 0 (its gradient term divides by beta_j)");
    return WAVE1D_OK;
}

// ---------------------------------------------------------------------------------------------
// Checkpoints of the march for the reverse pass: a header, then per checkpoint k (the state at
// step k * interval) the FP64 density ring, the S ring and the modes alpha, alpha'.  The float-pair
// density ring is rebuilt from the FP64 one on restore; the receiver history is not needed to
// march again.
// ---------------------------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int64_t M, K, W, ring, nsteps, interval, count, stride;
};
constexpr size_t kCkptHead = 256;

struct CkptPart {
    void* dev;
    size_t bytes;
};

std::vector<CkptPart> ckpt_parts(wave1d_plan_t p) {
    const Params& P = p->hp.P;
    const DevPlan& d = p->dp;
    const size_t K1 = (size_t)P.K + 1;
    return {{d.sig, sizeof(double) * (size_t)P.ring * P.M},
            {d.Sring, sizeof(double) * 2 * (size_t)P.W * K1},
            {d.alpha, sizeof(double) * 2 * K1},
            {d.alpha_p, sizeof(double) * 2 * K1}};
}

size_t ckpt_stride(wave1d_plan_t p) {
    size_t b = 0;
    for (const CkptPart& c : ckpt_parts(p)) b += (c.bytes + 255) / 256 * 256;
    return b;
}

void ckpt_header(wave1d_plan_t p, int64_t nsteps, int64_t interval, CkptHeader& h) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "WAVE1DC", 8);
    const Params& P = p->hp.P;
    h.M = P.M;
    h.K = P.K;
    h.W = P.W;
    h.ring = P.ring;
    h.nsteps = nsteps;
    h.interval = interval;
    h.count = (nsteps + interval - 1) / interval;
    h.stride = (int64_t)ckpt_stride(p);
}

// queue copies between the plan's march state and checkpoint k of buf (save: state -> buf)
int ckpt_copy(wave1d_plan_t p, char* buf, int64_t k, bool save) {
    char* at = buf + kCkptHead + (size_t)k * ckpt_stride(p);
    for (const CkptPart& c : ckpt_parts(p)) {
        if (save) CK(cudaMemcpyAsync(at, c.dev, c.bytes, cudaMemcpyDeviceToDevice, p->s));
        else CK(cudaMemcpyAsync(c.dev, at, c.bytes, cudaMemcpyDeviceToDevice, p->s));
        at += (c.bytes + 255) / 256 * 256;
    }
    return WAVE1D_OK;
}

// the march state of a plan (every part wave1d_state_save writes), kept on the device
struct DeviceState {
    std::vector<void*> bufs;
    int64_t n = 0;
    ~DeviceState() {
        for (void* b : bufs) cudaFree(b);
    }
};
}  // namespace

extern "C" {

int wave1d_adjoint(wave1d_plan_t p, int64_t nsteps, const double* sigma, const double* g, const double* ubar,
                   double* grad_beta, double* grad_g) {
    if (!p || !sigma) return fail(WAVE1D_EINVAL, "need a plan and sigma");
    int rc = adjoint_checks(p, nsteps, ubar, grad_beta, grad_g);
    if (rc) return rc;
    if ((rc = enter(p))) return rc;
    Reverse r;
    if ((rc = r.init(p))) return rc;
    if ((rc = r.steps(nsteps, 0, sigma, 0, g, ubar, grad_beta != nullptr, grad_g))) return rc;
    if ((rc = r.finish(grad_beta))) return rc;
    return leave(p);
}

int wave1d_checkpoint_size(wave1d_plan_t p, int64_t nsteps, int64_t interval, size_t* bytes) {
    if (!p || !bytes || nsteps < 1 || interval < 1) return fail(WAVE1D_EINVAL, "bad arguments");
    CkptHeader h;
    ckpt_header(p, nsteps, interval, h);
    *bytes = kCkptHead + (size_t)h.count * (size_t)h.stride;
    return WAVE1D_OK;
}

int wave1d_solve_checkpointed(wave1d_plan_t p, int64_t nsteps, int64_t interval, double* u_rec, int u_on_device,
                              void* ckpt, size_t bytes) {
    if (!p || !ckpt || nsteps < 1 || interval < 1) return fail(WAVE1D_EINVAL, "bad arguments");
    if (p->n != 0) return fail(WAVE1D_EINVAL, "the checkpointed march starts at step 0 (a fresh or reloaded plan)");
    if (nsteps > p->hp.P.Nt) return fail(WAVE1D_EDONE, "nsteps beyond the Nt of the plan");
    size_t need = 0;
    wave1d_checkpoint_size(p, nsteps, interval, &need);
    if (bytes < need) return fail(WAVE1D_EINVAL, "checkpoint buffer smaller than wave1d_checkpoint_size");
    int rc = enter(p);
    if (rc) return rc;
    CkptHeader h;
    ckpt_header(p, nsteps, interval, h);
    CK(cudaMemcpy(ckpt, &h, sizeof(h), cudaMemcpyHostToDevice));
    const int64_t R = p->hp.P.R;
    for (int64_t k = 0; k < h.count; k++) {
        if ((rc = ckpt_copy(p, (char*)ckpt, k, true))) return rc;
        const int64_t n0 = k * interval, cnt = std::min(interval, nsteps - n0);
        if ((rc = solve_steps(p, cnt, u_rec ? u_rec + n0 * R : nullptr, nullptr, u_on_device))) return rc;
    }
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

int wave1d_adjoint_checkpointed(wave1d_plan_t p, int64_t nsteps, int64_t interval, const void* ckpt, size_t bytes,
                                const double* ubar, double* grad_beta, double* grad_g) {
    if (!p || !ckpt || interval < 1) return fail(WAVE1D_EINVAL, "bad arguments");
    int rc = adjoint_checks(p, nsteps, ubar, grad_beta, grad_g);
    if (rc) return rc;
    size_t need = 0;
    wave1d_checkpoint_size(p, nsteps, interval, &need);
    if (bytes < need) return fail(WAVE1D_EINVAL, "checkpoint buffer smaller than wave1d_checkpoint_size");
    CkptHeader h, mine;
    ckpt_header(p, nsteps, interval, mine);
    if (cudaMemcpy(&h, ckpt, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess || std::memcmp(&h, &mine, sizeof(h)) != 0)
        return fail(WAVE1D_EINVAL, "not checkpoints of this plan, nsteps and interval (wave1d_solve_checkpointed)");
    if (p->n != nsteps) return fail(WAVE1D_EINVAL, "the plan is not at the step its checkpointed march ended on");
    if ((rc = enter(p))) return rc;
    const Params& P = p->hp.P;
    const int64_t M = P.M;
    // the march's final state, put back at the end
    DeviceState fin;
    for (const StatePart& sp : state_parts(p)) {
        void* b = nullptr;
        if (cudaMalloc(&b, sp.bytes) != cudaSuccess) return fail(WAVE1D_ENOMEM, "final-state copy");
        fin.bufs.push_back(b);
        CK(cudaMemcpyAsync(b, sp.dev, sp.bytes, cudaMemcpyDeviceToDevice, p->s));
    }
    fin.n = p->n;
    Reverse r;
    if ((rc = r.init(p))) return rc;
    double* seg = nullptr;
    if ((rc = r.wk.zeros(&seg, (size_t)std::min(interval, nsteps) * M))) return rc;
    const unsigned gS = blocks_for((int64_t)P.ring * M, 256, (int64_t)p->sms * 8);
    for (int64_t k = h.count - 1; k >= 0; k--) {
        // restore checkpoint k, march its segment again recording the densities, then the
        // segment's reverse steps
        const int64_t n0 = k * interval, n1 = std::min(nsteps, n0 + interval);
        if ((rc = ckpt_copy(p, (char*)const_cast<void*>(ckpt), k, false))) return rc;
        k_ck_sig2<<<gS, 256, 0, p->s>>>((int64_t)P.ring * M, p->dp.sig, (float2*)p->dp.sig2);
        k_ck_step<<<1, 1, 0, p->s>>>(p->dp.step, n0);
        CK(cudaGetLastError());
        p->n = n0;
        if ((rc = solve_steps(p, n1 - n0, nullptr, seg, 1))) return rc;
        if ((rc = r.steps(n1, n0, seg, n0, nullptr, ubar, grad_beta != nullptr, grad_g))) return rc;
    }
    if ((rc = r.finish(grad_beta))) return rc;
    size_t i = 0;
    for (const StatePart& sp : state_parts(p))
        CK(cudaMemcpyAsync(sp.dev, fin.bufs[i++], sp.bytes, cudaMemcpyDeviceToDevice, p->s));
    k_ck_step<<<1, 1, 0, p->s>>>(p->dp.step, fin.n);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(p->s));
    p->n = fin.n;
    if ((rc = leave(p))) return rc;
    return check_status(p);
}

int wave1d_destroy(wave1d_plan_t p) {
    if (!p) return WAVE1D_OK;
    if (p->s) cudaStreamSynchronize(p->s);
    drop_graphs(p);
    for (int i = 0; i <= WAVE1D_NSTAGE; i++)
        if (p->prof_ev[i]) cudaEventDestroy(p->prof_ev[i]);
    if (p->nu_s) wave1d_nufft_destroy(p->nu_s);
    if (p->nu_r) wave1d_nufft_destroy(p->nu_r);
    for (void* a : p->allocs) cudaFree(a);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->s2) cudaStreamSynchronize(p->s2);
    if (p->s2) cudaStreamDestroy(p->s2);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
    return WAVE1D_OK;
}

}  // extern "C"
