// Per-step kernels of the WFP march.  One time step n -> n+1 is, in launch order:
//   k_local      local explicit sum over the last delta of history (Sec. 4.1, m >= 1)
//   k_spread     type-1 spreading of sigma^n onto the fine grid (eq. densco via NUFFT)
//   k_fft_cols / k_fft_rows   forward complex FFT of the grid viewed as L = nf/2 complex points
//   k_modes      S_k^n, FIR driving terms, exact rotation, type-2 spectrum (Sec. 3)
//   [k_rbc_grid, k_rbc_update]  radiation projection on projection steps (Sec. 4.4)
//   k_fft_cols / k_fft_rows   inverse FFT of the type-2 spectrum
//   k_interp     u_H at springs and receivers (eq. historySol1 via NUFFT)
//   k_solve      right-hand side and block solve of -(I + S) sigma^{n+1} = ... (eq. linearSystem)
//   k_receivers  u = u_L + u_H at receivers; the last block advances the step counter
// Kernels read the step index n from device memory so that captured graphs can be replayed.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "../../include/wave1d.h"

namespace wave1d {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ int ring_slot(int64_t q, int ring) {
    int64_t r = q % ring;
    return (int)(r < 0 ? r + ring : r);
}

__device__ __forceinline__ int64_t load_step(const DevPlan& P) {
    return *((const volatile int64_t*)P.step);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// type-1 spreading, gather form: G[i] = sum over springs whose support starts at c = i - t of
// sigma_j^n psi_{j,t}.  Deterministic (no atomics).
// ---------------------------------------------------------------------------------------------
__global__ void k_spread(DevPlan P) {
    int64_t n = load_step(P);
    int slot = ring_slot(n, P.ring);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nf; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < P.w; t++) {
            int c = i - t;
            if (c < 0) c += P.nf;
            int e1 = P.bin_ptr[c + 1];
            for (int e = P.bin_ptr[c]; e < e1; e++) {
                int j = P.bin_list[e];
                acc = fma(P.sig[(int64_t)j * P.ring + slot], P.sp_ker[(int64_t)j * P.w + t], acc);
            }
        }
        P.grid[i] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// Complex FFT of length L = L1 * L2 (powers of two), X[k] = sum_i z[i] e^{sign 2 pi i ik/L}:
//   columns: for each i2, FFT over i1 of z[i2 + L2 i1], times e^{sign 2 pi i i2 k1/L} -> Y[k1 L2 + i2]
//   rows:    for each k1, FFT over i2 of Y[k1 L2 + i2] -> X[k1 + L1 k2]
// Each block transforms one line in shared memory: bit-reversed load, radix-2 DIT stages.
// tw[j] = e^{+2 pi i j / L}.
// ---------------------------------------------------------------------------------------------
__device__ void fft_line(double2* a, int N, int logN, const double2* tw, int L, int sign) {
    for (int s = 1; s <= logN; s++) {
        int half = 1 << (s - 1);
        int step = L / (2 * half);
        for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
            int pos = j & (half - 1);
            int i0 = ((j >> (s - 1)) << s) + pos;
            int i1 = i0 + half;
            double2 w = tw[pos * step];
            if (sign < 0) w.y = -w.y;
            double2 t = cmul(w, a[i1]);
            double2 u = a[i0];
            a[i0] = cadd(u, t);
            a[i1] = csub(u, t);
        }
        __syncthreads();
    }
}

__global__ void k_fft_cols(const double2* __restrict__ in, double2* __restrict__ out,
                           const double2* __restrict__ tw, int L, int L1, int L2, int logL1, int sign) {
    extern __shared__ double2 sm[];
    int i2 = blockIdx.x;
    for (int i1 = threadIdx.x; i1 < L1; i1 += blockDim.x)
        sm[__brev(i1) >> (32 - logL1)] = in[i2 + (int64_t)L2 * i1];
    __syncthreads();
    fft_line(sm, L1, logL1, tw, L, sign);
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
    int k1 = blockIdx.x;
    for (int i2 = threadIdx.x; i2 < L2; i2 += blockDim.x)
        sm[__brev(i2) >> (32 - logL2)] = in[(int64_t)k1 * L2 + i2];
    __syncthreads();
    fft_line(sm, L2, logL2, tw, L, sign);
    for (int k2 = threadIdx.x; k2 < L2; k2 += blockDim.x) out[k1 + (int64_t)L1 * k2] = sm[k2];
}

// ---------------------------------------------------------------------------------------------
// Type-2 spectrum of mode k for the inverse real FFT: F'_k = deconv2_k alpha_k;
// Zs[k] = F'_k (1 + i w^k), Zs[L-k] = conj(F'_k) (1 - i w^{L-k}), w = e^{-2 pi i / nf}.
// (Entries with K < idx < L - K stay zero.)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void write_type2(const DevPlan& P, int k, double2 a, double2* Zs) {
    double d2 = P.deconv2[k];
    double2 F = make_double2(d2 * a.x, d2 * a.y);
    double s, c;
    sincospi(-2.0 * (double)k / (double)P.nf, &s, &c);          // w^k
    double2 iw = make_double2(-s, c);                            // i w^k
    Zs[k] = cadd(F, cmul(F, iw));
    if (k > 0) {
        int kk = P.L - k;
        sincospi(-2.0 * (double)kk / (double)P.nf, &s, &c);
        double2 iw2 = make_double2(-s, c);
        double2 Fc = cconj(F);
        Zs[kk] = csub(Fc, cmul(Fc, iw2));
    }
}

// ---------------------------------------------------------------------------------------------
// Modes: four threads per mode k.
//   S_k^n = deconv1_k F_k, F_k = E_k + e^{2 pi i k/nf} O_k from the half-length FFT Z
//   (E = (Z_k + conj Z_{L-k})/2, O = (Z_k - conj Z_{L-k})/(2i)), stored in ring slot n mod W;
//   h_k = sum_m dt p_k(m dt) S_k^{n-m}, g_k likewise (eq. hkcompdisc);
//   alpha, alpha' rotated and driven (eq. alphakEvolutionFormulas); type-2 spectrum written.
// ---------------------------------------------------------------------------------------------
__global__ void k_modes(DevPlan P) {
    int64_t n = load_step(P);
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    int k = tid >> 2, q = tid & 3;
    bool valid = k <= P.K;
    int kk = valid ? k : P.K;
    const double2* Z = (const double2*)P.spec;
    double2 zk = Z[kk];
    double2 zm = Z[kk == 0 ? 0 : P.L - kk];
    double2 E = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
    double2 D = make_double2(0.5 * (zk.x - zm.x), 0.5 * (zk.y + zm.y));
    double2 O = make_double2(D.y, -D.x);
    double s, c;
    sincospi(2.0 * (double)kk / (double)P.nf, &s, &c);
    double2 F = cadd(E, cmul(make_double2(c, s), O));
    double d1 = P.deconv1[kk];
    double2 Sn = make_double2(d1 * F.x, d1 * F.y);
    int K1 = P.K + 1;
    double2* Sring = (double2*)P.Sring;
    const double2* pq = (const double2*)P.pq;
    double2 h = make_double2(0.0, 0.0), g = make_double2(0.0, 0.0);
    for (int m = q; m < P.W; m += 4) {
        double2 Sm;
        if (m == 0) {
            Sm = Sn;
        } else {
            int slot = ring_slot(n - m, P.W);
            Sm = Sring[(int64_t)slot * K1 + kk];
        }
        double2 w = pq[(int64_t)m * K1 + kk];
        h.x = fma(w.x, Sm.x, h.x);
        h.y = fma(w.x, Sm.y, h.y);
        g.x = fma(w.y, Sm.x, g.x);
        g.y = fma(w.y, Sm.y, g.y);
    }
    for (int o = 1; o < 4; o <<= 1) {
        h.x += __shfl_xor_sync(0xffffffffu, h.x, o);
        h.y += __shfl_xor_sync(0xffffffffu, h.y, o);
        g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
    }
    if (!valid || q != 0) return;
    Sring[(int64_t)ring_slot(n, P.W) * K1 + k] = Sn;
    double2* al = (double2*)P.alpha;
    double2* alp = (double2*)P.alpha_p;
    double2 a = al[k], ap = alp[k];
    double cs = P.rot[3 * k], so = P.rot[3 * k + 1], ks = P.rot[3 * k + 2];
    double2 an = make_double2(fma(a.x, cs, fma(ap.x, so, h.x)), fma(a.y, cs, fma(ap.y, so, h.y)));
    double2 apn = make_double2(fma(ap.x, cs, fma(-a.x, ks, g.x)), fma(ap.y, cs, fma(-a.y, ks, g.y)));
    al[k] = an;
    alp[k] = apn;
    write_type2(P, k, an, (double2*)P.spec2);
}


// ---------------------------------------------------------------------------------------------
// Radiation projection (Sec. 4.4), applied to alpha^{n+1}, alpha'^{n+1} on projection steps.
// The 2K-point grid values of the real field with modes |k| <= K-1 change only at the 4W points
// next to x = +-pi, so the projected coefficients are
//   alpha_k + (1/2K) sum_{i in I} du_i e^{+i k x_i},  alpha'_k + (1/2K) sum_{i in I} dv_i e^{+i k x_i}
// with du = (phi_s - 1) u, dv = phi_s' u + (phi_s - 1) v (eq. vtilde), and alpha_K = 0.
// x_i = i pi/K, so e^{i k x_i} = e^{i pi (k i mod 2K)/K} (exact argument reduction).
// ---------------------------------------------------------------------------------------------
__global__ void k_rbc_grid(DevPlan P) {
    int pt = blockIdx.x;                     // one block per rolled-off grid point
    int ig = P.rbc_idx[pt];
    const double2* al = (const double2*)P.alpha;
    const double2* alp = (const double2*)P.alpha_p;
    double su = 0.0, sv = 0.0;
    int64_t twoK = 2 * (int64_t)P.K;
    for (int k = 1 + threadIdx.x; k < P.K; k += blockDim.x) {
        int64_t a = ((int64_t)k * ig) % twoK;
        double s, c;
        sincospi((double)a / (double)P.K, &s, &c);            // e^{+i k x}; use conj for e^{-ikx}
        double2 e = make_double2(c, -s);
        su += cmul(al[k], e).x;
        sv += cmul(alp[k], e).x;
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
    double2 a, ap;
    if (k == P.K) {
        a = make_double2(0.0, 0.0);
        ap = a;
    } else {
        double2 du = make_double2(0.0, 0.0), dv = make_double2(0.0, 0.0);
        int64_t twoK = 2 * (int64_t)P.K;
        for (int pt = 0; pt < npts; pt++) {
            int64_t ang = ((int64_t)k * P.rbc_idx[pt]) % twoK;
            double s, c;
            sincospi((double)ang / (double)P.K, &s, &c);
            double xu = P.rbc_uv[4 * pt + 2], xv = P.rbc_uv[4 * pt + 3];
            du.x = fma(xu, c, du.x);
            du.y = fma(xu, s, du.y);
            dv.x = fma(xv, c, dv.x);
            dv.y = fma(xv, s, dv.y);
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

// ---------------------------------------------------------------------------------------------
// type-2 interpolation: u_H(x_t) = sum_{t'} G'[(i0 + t') mod nf] psi_{t,t'} for springs, then
// receivers.
// ---------------------------------------------------------------------------------------------
__global__ void k_interp(DevPlan P) {
    int64_t total = P.M + P.R;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        bool spring = t < P.M;
        int64_t j = spring ? t : t - P.M;
        int i0 = spring ? P.sp_i0[j] : P.rc_i0[j];
        const double* ker = spring ? P.sp_ker + j * P.w : P.rc_ker + j * P.w;
        double acc = 0.0;
        int i = i0;
        for (int tt = 0; tt < P.w; tt++) {
            acc = fma(P.grid[i], ker[tt], acc);
            i = (i + 1 == P.nf) ? 0 : i + 1;
        }
        if (spring) P.uH[j] = acc;
        else P.uHr[j] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// local explicit sum (Sec. 4.1, eq. periodicIE_disc, m >= 1): one warp per target spring
//   c_j = sum_{l in N_delta(x_j)} sum_{m} Q_m(d_jl) sigma_l^{n+1-m}
// ---------------------------------------------------------------------------------------------
__global__ void k_local(DevPlan P) {
    int64_t n = load_step(P);
    int lane = threadIdx.x & 31;
    int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (j >= P.M) return;
    double acc = 0.0;
    int64_t e1 = P.row_ptr[j + 1];
    for (int64_t e = P.row_ptr[j] + lane; e < e1; e += 32) {
        int l = P.src[e];
        int mr = P.mrange[e];
        int mlo = mr & 0xffff, cnt = mr >> 16;
        const double* wq = P.wq + P.woff[e];
        const double* sl = P.sig + (int64_t)l * P.ring;
        int slot = ring_slot(n + 1 - mlo, P.ring);
        for (int c = 0; c < cnt; c++) {
            acc = fma(wq[c], sl[slot], acc);
            slot = (slot == 0) ? P.ring - 1 : slot - 1;
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) P.clocal[j] = acc;
}

// incident forcing g_j(t) = beta_j f(x_j - t), f periodised over 2 pi in the periodic box (eq. gj)
__device__ double incident(const DevPlan& P, double s) {
    double f = 0.0;
    const double kTwoPi = 6.283185307179586476925286766559;
    for (int i = 0; i < P.npulse; i++) {
        double amp = P.pulse[3 * i], cen = P.pulse[3 * i + 1], wid = P.pulse[3 * i + 2];
        if (P.bc == WAVE1D_FREE) {
            double z = (s - cen) / wid;
            if (fabs(z) <= 40.0) f += amp * exp(-0.5 * z * z);
        } else {
            double span = 40.0 * wid;
            int64_t m0 = (int64_t)floor((cen - s - span) / kTwoPi);
            int64_t m1 = (int64_t)ceil((cen - s + span) / kTwoPi);
            for (int64_t m = m0; m <= m1; m++) {
                double z = (s + kTwoPi * (double)m - cen) / wid;
                if (fabs(z) <= 40.0) f += amp * exp(-0.5 * z * z);
            }
        }
    }
    return f;
}

// right-hand side of eq. linearSystem: rhs_j = -g_j - (beta_j/2) c_j - beta_j u_H(x_j)
__global__ void k_rhs(DevPlan P) {
    int64_t n = load_step(P);
    double t1 = (double)(n + 1) * P.dt;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M;
         j += (int64_t)gridDim.x * blockDim.x) {
        double bj = P.beta[j];
        double g = P.g_ext ? P.g_ext[j] : bj * incident(P, P.x[j] - t1);
        P.rhs[j] = -g - 0.5 * bj * P.clocal[j] - bj * P.uH[j];
    }
}

// block solve sigma^{n+1} = (I + S)^{-1} rhs, one warp per block of springs closer than dt
__global__ void k_solve(DevPlan P) {
    int64_t n = load_step(P);
    int lane = threadIdx.x & 31;
    int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= P.nblocks) return;
    int64_t m0 = P.blk_ptr[b];
    int s = (int)(P.blk_ptr[b + 1] - m0);
    const double* inv = P.inv + P.blk_inv_off[b];
    int slot = ring_slot(n + 1, P.ring);
    for (int i = lane; i < s; i += 32) {
        double acc = 0.0;
        for (int l = 0; l < s; l++) acc = fma(inv[(int64_t)i * s + l], P.rhs[P.blk_members[m0 + l]], acc);
        int j = P.blk_members[m0 + i];
        P.sig[(int64_t)j * P.ring + slot] = acc;
        if (!isfinite(acc)) atomicExch(P.status, (int)WAVE1D_ENONFINITE);
        if (P.sig_hist) P.sig_hist[(n % P.chunk) * P.M + P.perm[j]] = acc;
    }
}

// receivers: u = 1/2 sum_l sum_{m>=0} Q_m sigma_l^{n+1-m} + u_H(x_r); the block that finishes last
// advances the step counter (every other block has read n before it counts itself done).
__global__ void k_receivers(DevPlan P) {
    int64_t n = load_step(P);
    int lane = threadIdx.x & 31;
    int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r < P.R) {
        double acc = 0.0;
        int64_t e1 = P.rrow_ptr[r + 1];
        for (int64_t e = P.rrow_ptr[r] + lane; e < e1; e += 32) {
            int l = P.rsrc[e];
            int mr = P.rmrange[e];
            int mlo = mr & 0xffff, cnt = mr >> 16;
            const double* wq = P.rwq + P.rwoff[e];
            const double* sl = P.sig + (int64_t)l * P.ring;
            int slot = ring_slot(n + 1 - mlo, P.ring);
            for (int c = 0; c < cnt; c++) {
                acc = fma(wq[c], sl[slot], acc);
                slot = (slot == 0) ? P.ring - 1 : slot - 1;
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) P.rec_hist[(n % P.chunk) * P.R + r] = 0.5 * acc + P.uHr[r];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long done = atomicAdd((unsigned long long*)&P.step[1], 1ull);
        if (done == gridDim.x - 1) {
            P.step[1] = 0;
            __threadfence();
            P.step[0] = n + 1;
        }
    }
}

// caller-order gathers and scatters
__global__ void k_sigma_to_caller(DevPlan P, int64_t q, double* out) {
    int slot = ring_slot(q, P.ring);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x)
        out[P.perm[j]] = P.sig[j * P.ring + slot];
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
