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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "batch_host.h"
#include "internal.h"
#include "phases.cuh"
#include "../../include/wave1d.h"

namespace wave1d {
__global__ void k_local_items(DevPlan P);
__global__ void k_solve(DevPlan P);
__global__ void k_mx_gather(DevPlan P, const int64_t* perm, double* c);
__global__ void k_mx_receivers(int64_t R, const int64_t* perm, const double* u, double* uHr);

// forward FFT column pass of every instance's fine grid (blockIdx.y = instance): for column i2,
// FFT over i1 of z[i2 + L2 i1] (sign +), times e^{+2 pi i i2 k1 / L}  ->  Y[k1 L2 + i2]
__global__ void k_bfft_cols(const double2* __restrict__ grids, double2* __restrict__ Ys,
                            const double2* __restrict__ tw, int L, int L1, int L2, int logL1) {
    extern __shared__ double2 sm[];
    double2* twN = sm + L1;
    const int i2 = blockIdx.x;
    const double2* in = grids + (int64_t)blockIdx.y * L;
    double2* out = Ys + (int64_t)blockIdx.y * L;
    for (int j = threadIdx.x; j < L1 / 2; j += blockDim.x) twN[j] = tw[j * (L / L1)];
    for (int i1 = threadIdx.x; i1 < L1; i1 += blockDim.x) sm[__brev(i1) >> (32 - logL1)] = in[i2 + (int64_t)L2 * i1];
    __syncthreads();
    fft_lines(sm, nullptr, twN, L1, logL1);
    for (int k1 = threadIdx.x; k1 < L1; k1 += blockDim.x)
        out[(int64_t)k1 * L2 + i2] = cmul(sm[k1], tw[((int64_t)i2 * k1) & (L - 1)]);
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
__global__ void k_b_rhs(DevPlan P, const int64_t* __restrict__ perm, const double* __restrict__ u,
                        const int32_t* __restrict__ inst_of, const double* __restrict__ pulse) {
    const int64_t n = load_step(P);
    const double kTwoPi = 6.283185307179586476925286766559;
    const double kInvTwoPi = 0.15915494309189533576888376337251;
    const double t = (double)(n + 1) * P.dt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.M; i += (int64_t)gridDim.x * blockDim.x) {
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
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0, sms = 1, B = 0, chunk = 32;
    int64_t n = 0;
    wave1d_nufft_t nu_s = nullptr, nu_r = nullptr;
    int64_t *perm_s = nullptr, *perm_r = nullptr;
    int32_t* inst_of = nullptr;
    double *pulse = nullptr, *c = nullptr, *u = nullptr, *ur = nullptr, *grids = nullptr, *work = nullptr,
           *sig_hist = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step without / with the density history
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

// queue one step of every instance
int enqueue_batch_step(wave1d_batch_t p, double* sig_hist) {
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
    if (o.local_weights != 0)
        return bfail(WAVE1D_EINVAL, "the batched march stores its local weights (local_weights = 0)");
    if (o.max_block <= 0) o.max_block = 4096;
    if (o.max_local_bytes <= 0) o.max_local_bytes = (int64_t)16 << 30;

    wave1d_batch_t p = new (std::nothrow) wave1d_batch_s();
    if (!p) return bfail(WAVE1D_ENOMEM, "host allocation");
    auto cleanup = [&](int code) {
        wave1d_batch_destroy(p);
        return code;
    };
    p->B = n_inst;
    // the instances' own tables, then joined
    std::vector<HostPlan> inst((size_t)n_inst);
    std::string err;
    int64_t bytes = 0;
    for (int b = 0; b < n_inst; b++) {
        const int64_t M = offsets[b + 1] - offsets[b];
        int rc = build_host_plan(x + offsets[b], beta + offsets[b], M, WAVE1D_PERIODIC, dt, Nt, tol, o.p, o.gamma, o.W,
                                 o.NL, o.Ng, 0, o.rbc_period, o.max_block, o.max_local_bytes - bytes, inst[b], err);
        if (rc == WAVE1D_OK) {
            double none = 0.0;
            const int64_t R = r_offsets ? r_offsets[b + 1] - r_offsets[b] : 0;
            rc = build_receivers(inst[b], R ? xr + r_offsets[b] : &none, R, err);
        }
        if (rc) return cleanup(bfail(rc, "instance " + std::to_string(b) + ": " + err));
        bytes += (int64_t)inst[b].litems.w.size() * 4;
    }
    if (int rc = join_instances(inst, p->bt, err)) return cleanup(bfail(rc, err));
    inst.clear();
    const Params& P = p->bt.g.P;
    p->user = (cudaStream_t)o.stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) return cleanup(bfail(WAVE1D_ECUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(bfail(WAVE1D_ECUDA, "stream/event creation failed"));
    if (cudaEventRecord(p->ev_in, p->user) != cudaSuccess || cudaStreamWaitEvent(p->s, p->ev_in, 0) != cudaSuccess)
        return cleanup(bfail(WAVE1D_ECUDA, "stream ordering failed"));
    int rc;
    if ((rc = upload_joined(p)) || (rc = upload_views(p))) return cleanup(rc);
    std::vector<double> pl((size_t)3 * n_inst);
    for (int b = 0; b < n_inst; b++) {
        pl[3 * b] = pulse[3 * b];
        pl[3 * b + 1] = pulse[3 * b + 1];
        pl[3 * b + 2] = 1.0 / pulse[3 * b + 2];
    }
    if ((rc = bupload(p, pl, &p->pulse)) || (rc = bupload(p, p->bt.inst_of, &p->inst_of))) return cleanup(rc);
    if ((rc = balloc(p, &p->c, (size_t)P.M)) || (rc = balloc(p, &p->u, (size_t)P.M))) return cleanup(rc);
    // batched NUFFT plans of the springs and of the receivers: the instances' fine grids, kernel
    // (width from tol, as each instance's plan) and deconvolution
    rc = wave1d_nufft_plan_many(p->bt.g.x.data(), p->bt.moff.data(), n_inst, P.K, tol, 0, (void*)p->s, &p->nu_s);
    if (rc) return cleanup(bfail(rc, std::string("batched NUFFT plan: ") + wave1d_nufft_strerror()));
    std::vector<int64_t> perm((size_t)P.M);
    if ((rc = wave1d_nufft_perm(p->nu_s, perm.data()))) return cleanup(bfail(rc, wave1d_nufft_strerror()));
    if ((rc = bupload(p, perm, &p->perm_s))) return cleanup(rc);
    if (P.R > 0) {
        rc = wave1d_nufft_plan_many(p->bt.g.xr.data(), p->bt.roff.data(), n_inst, P.K, tol, 0, (void*)p->s, &p->nu_r);
        if (rc) return cleanup(bfail(rc, std::string("batched NUFFT plan of the receivers: ") + wave1d_nufft_strerror()));
        std::vector<int64_t> permr((size_t)P.R);
        if ((rc = wave1d_nufft_perm(p->nu_r, permr.data()))) return cleanup(bfail(rc, wave1d_nufft_strerror()));
        if ((rc = bupload(p, permr, &p->perm_r)) || (rc = balloc(p, &p->ur, (size_t)P.R))) return cleanup(rc);
    }
    if (cudaFuncSetAttribute(k_bhist_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_phase_smem(P.L2)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_bfft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem_bytes(P.L1)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_bhist_icols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)icols_phase_smem(P.L1)) !=
            cudaSuccess)
        return cleanup(bfail(WAVE1D_ECUDA, "cannot size the shared memory of the history passes"));
    if (cudaStreamSynchronize(p->s) != cudaSuccess) return cleanup(bfail(WAVE1D_ECUDA, "plan upload failed"));
    // the device holds the joined weights now: release the host copies
    std::vector<float>().swap(p->bt.g.litems.w);
    std::vector<float>().swap(p->bt.g.ritems.w);
    std::vector<double>().swap(p->bt.g.inv);
    *out = p;
    return WAVE1D_OK;
}

int wave1d_batch_solve(wave1d_batch_t p, int64_t nsteps, double* u_rec, double* sigma, int out_on_device) {
    if (!p || nsteps < 0) return bfail(WAVE1D_EINVAL, "bad solve arguments");
    const Params& P = p->bt.g.P;
    if (p->n + nsteps > P.Nt) return bfail(WAVE1D_EDONE, "nsteps beyond the Nt of the plan");
    BCK(cudaSetDevice(p->device));
    BCK(cudaEventRecord(p->ev_in, p->user));
    BCK(cudaStreamWaitEvent(p->s, p->ev_in, 0));
    if (sigma && !p->sig_hist) {
        int rc = balloc(p, &p->sig_hist, (size_t)p->chunk * P.M);
        if (rc) return rc;
    }
    cudaGraphExec_t& ge = p->graph[sigma ? 1 : 0];
    if (!ge) {
        cudaGraph_t graph;
        BCK(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_batch_step(p, sigma ? p->sig_hist : nullptr);
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
            if (u_rec && P.R > 0)
                BCK(cudaMemcpyAsync(u_rec + first * P.R, p->g.rec_hist + slot0 * P.R, pending * P.R * sizeof(double),
                                    kind, p->s));
            if (sigma)
                BCK(cudaMemcpyAsync(sigma + first * P.M, p->sig_hist + slot0 * P.M, pending * P.M * sizeof(double),
                                    kind, p->s));
            pending = 0;
        }
    }
    BCK(cudaEventRecord(p->ev_out, p->s));
    BCK(cudaStreamWaitEvent(p->user, p->ev_out, 0));
    int st = 0;
    BCK(cudaMemcpyAsync(&st, p->g.status, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    BCK(cudaStreamSynchronize(p->s));
    if (st != 0) return bfail(st, "a density became non-finite during the march");
    return WAVE1D_OK;
}

int wave1d_batch_destroy(wave1d_batch_t p) {
    if (!p) return WAVE1D_OK;
    if (p->s) cudaStreamSynchronize(p->s);
    for (auto& g : p->graph)
        if (g) cudaGraphExecDestroy(g);
    if (p->nu_s) wave1d_nufft_destroy(p->nu_s);
    if (p->nu_r) wave1d_nufft_destroy(p->nu_r);
    for (void* a : p->allocs) cudaFree(a);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
    return WAVE1D_OK;
}

const char* wave1d_batch_strerror(void) { return g_batch_error.c_str(); }

}  // extern "C"
