// Time step of plans opened with opts.local_weights = 1: no per-pair data on the device.  The
// springs are sorted, so the sources within delta of a target are an index window, and the local
// weights Q_m(d) (Sec. 4.1) come from their polynomials in the distance (range.cuh).  One step:
//
//   k_rs_local      local explicit sum c_j over m >= 1 (Sec. 4.1), compensated FP32 pairs
//   history pipeline (type-1 NUFFT, mode update, [projection], type-2 NUFFT): the per-stage
//                   kernels of every plan; the interpolation leaves rhs_j = -g_j - beta_j u_H(x_j)
//   k_rs_solve_init rhs_j -= (beta_j / 2) c_j; first iterate extrapolated from sigma^{n-7..n}
//   k_rs_jacobi     Jacobi sweeps of (I + S) sigma^{n+1} = rhs (eq. linearSystem), S_jl =
//                   (beta_j / 2) Q_0(d_jl) over the sources closer than dt, until the largest
//                   change is below kRsTol of the largest density (launches after that return at
//                   once, so the step is a fixed sequence of launches and can be captured)
//   k_rs_store      sigma^{n+1} into the rings (status WAVE1D_ENOTCONV if no sweep converged)
//   k_rs_receivers  u_L at the receivers (eq. localSol2, all m including m = 0), FP64
//   k_rs_finish     u = u_L + u_H at the receivers, step counter
//
// Every kernel reads the step index from the device counter (graphs of steps are replayed).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phases.cuh"
#include "range.cuh"
#include "../../include/wave1d.h"

namespace wave1d {

namespace {
constexpr double kPiR = 3.14159265358979323846264338327950288;
constexpr int kRsChunk = 32;      // sources per chunk (one per lane of warp 0 in the set-up)
constexpr int kRsIvCap = 32;      // intervals whose e-vectors are held at once (3 blocks of 256 threads per SM)
// one interval's row of e-vector records: 32 records of 12 floats and 4 floats of padding, so the
// rows of consecutive intervals start 4 banks apart (threads of a warp read the records of the 2-3
// intervals their distances fall in)
constexpr int kRsRow = kRsChunk * rs::kERecord + 4;
}  // namespace

// shared memory of k_rs_local (bytes): e-vector rows, the chunk's densities, the interval table
size_t rs_local_smem(int nint, int nm) {
    return (size_t)kRsIvCap * kRsRow * sizeof(float) + (size_t)nm * kRsChunk * sizeof(float2) +
           (size_t)4 * nint * sizeof(float);
}

// position of extended source index e: the same expression as the host's window tests
__device__ __forceinline__ double rs_xext(const DevPlan& P, int64_t e) {
    if (e < 0) return P.x[e + P.M] - 2.0 * kPiR;
    if (e >= P.M) return P.x[e - P.M] + 2.0 * kPiR;
    return P.x[e];
}

__device__ __forceinline__ int64_t rs_spring(int64_t e, int64_t M) { return e < 0 ? e + M : (e >= M ? e - M : e); }

// interval of an FP64 distance
__device__ __forceinline__ int rs_locate64(const RangeDev& R, double d) {
    int lo = 0, hi = R.nint;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (d < __ldg(R.bp + mid)) hi = mid;
        else lo = mid;
    }
    return lo;
}

// Chebyshev series of degree 7 (Clenshaw), FP64
__device__ __forceinline__ double rs_cheb(const double* c, double z) {
    double b0 = 0.0, b1 = 0.0;
    for (int r = 7; r >= 1; r--) {
        const double b2 = b1;
        b1 = b0;
        b0 = fma(2.0 * z, b1, __ldg(c + r) - b2);
    }
    return fma(z, b0, __ldg(c) - b1);
}

// Q_0(d) from its series (zero at d >= dt, where m_min = 1)
__device__ __forceinline__ double rs_q0(const RangeDev& R, double d) {
    const int iv = rs_locate64(R, d);
    if (iv >= R.iv_dt) return 0.0;
    const double z = (d - __ldg(R.mid + iv)) * (double)__ldg(R.ih + iv);
    return rs_cheb(R.cheb + (size_t)iv * R.nm * 8, z);
}

// ---------------------------------------------------------------------------------------------
// Local explicit sum, one block per kRsTargets consecutive targets (thread t: target j0 + t).
// The block's sources (window [wlo, whi) of extended indices) are visited twice over as
// "left" sources (strictly left of the target: d = x_j - x_e) and "right" sources (at or right
// of it: d = x_e - x_j), in chunks of 32.  Per chunk:
//   1. once per 8 chunks, one thread per source: its position on the block grid (range.cuh) and
//      the interval range its distances to the block's targets fall in;
//   2. the chunk's densities sigma^{n+1-m}, m = 1 .. m_max, into shared memory;
//   3. for each interval of the chunk's range (at most kRsIvCap at a time), one warp folds the
//      densities of all 32 sources into their e-vectors (coefficients are warp-uniform loads);
//   4. each thread walks the 32 sources: z on the tracked interval of the side (it moves by about
//      one interval from one source to the next), and the polynomial of the source's e-vector at z
//      into the thread's compensated accumulator.
// Which side counts a source is decided by index: e < lb_j (the first spring at x_j's position) is
// strictly left.  Q_m is continuous across the breakpoints other than dt, so a pair within
// rounding of one takes either neighbouring interval's polynomial; at dt the spring's FP64 window
// of near sources decides (near_side in range.cuh).
// ---------------------------------------------------------------------------------------------
template <int S>
__device__ __forceinline__ void rs_pairs(const float* sE, const float4* sMeta, const float* ivt, const int* cell,
                                         float cscale, int nint, int iv_dt, int k0, int k1, int W0, int W1, int lbj,
                                         int nbl, int nbc, float bh, float bl, rs::Track& tr, float& a0h, float& a0l,
                                         float& a1h, float& a1l) {
    for (int k = k0; k < k1; k += 2) {
        // the record and z of sources k and k + 1 (null where the pair does not count in this
        // window), then both polynomials as independent chains.  z is computed for every slot
        // (the group's meta holds 256 defined entries, so slot k + 1 >= k1 reads one); only a
        // pair that counts moves the tracked interval.
        const float* rec[2];
        float zh[2], zl[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int kk = k + u;
            const float4 mt = sMeta[kk];
            const int e = __float_as_int(mt.z), lohi = __float_as_int(mt.w);
            const int lo = max(lohi & 0x7fff, W0), hi = min(lohi >> 16, W1);
            const bool valid = kk < k1 && lo <= hi && (S < 0 ? e < lbj : e >= lbj);
            float h0, l0;
            rs::z_of<S>(tr, mt.x, mt.y, h0, l0);
            if (valid && fabsf(h0) > rs::kZTol) rs::walk<S>(ivt, cell, cscale, nint, bh, bl, mt.x, mt.y, tr, h0, l0);
            if (valid && (lohi & 0x8000))
                rs::near_side<S>(ivt, iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt.x, mt.y, tr, h0, l0);
            const bool ok = valid && fabsf(h0) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi;
            rec[u] = ok ? sE + (tr.iv - W0) * kRsRow + kk * rs::kERecord : nullptr;
            zh[u] = h0;
            zl[u] = l0;
        }
        if (rec[0]) rs::evec_eval(rec[0], zh[0], zl[0], a0h, a0l);
        if (rec[1]) rs::evec_eval(rec[1], zh[1], zl[1], a1h, a1l);
    }
}

// The pairs of one side for one target in a chunk whose interval range takes several windows of
// e-vectors: the sources in walk order (right: k ascending; left: k descending, so the distance
// grows along both) from the thread's cursor cur, evaluated in the window that holds their
// interval.  A source whose interval lies beyond the window stops the walk there (the tracked
// interval kept, the cursor on it) until the next window; so each source is walked once per
// thread and chunk, not once per window.  Sources beyond delta end the side.  k0 .. k1 - 1: the
// side's sources in the chunk; par alternates the two accumulators.
template <int S>
__device__ __forceinline__ void rs_pairs_cursor(const float* sE, const float4* sMeta, const float* ivt, const int* cell,
                                                float cscale, int nint, int iv_dt, int k0, int k1, int& cur, int W0,
                                                int W1, int lbj, int nbl, int nbc, float bh, float bl, rs::Track& tr,
                                                int& par, float& a0h, float& a0l, float& a1h, float& a1l) {
    while (S > 0 ? cur < k1 : cur >= k0) {
        const int k = cur;
        const float4 mt = sMeta[k];
        const int e = __float_as_int(mt.z), lohi = __float_as_int(mt.w);
        const int lo = lohi & 0x7fff, hi = lohi >> 16;
        if (lo > hi || (S < 0 ? e >= lbj : e < lbj)) {
            cur += S;
            continue;
        }
        if (lo > W1) break;                                   // its interval lies in a later window
        float zh, zl;
        rs::z_of<S>(tr, mt.x, mt.y, zh, zl);
        if (fabsf(zh) > rs::kZTol) rs::walk<S>(ivt, cell, cscale, nint, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt, iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (tr.iv > W1 && fabsf(zh) <= rs::kZTol) break;     // a later window
        if (fabsf(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi && tr.iv >= W0) {
            const float* rec = sE + (tr.iv - W0) * kRsRow + k * rs::kERecord;
            if (par) rs::evec_eval(rec, zh, zl, a1h, a1l);
            else rs::evec_eval(rec, zh, zl, a0h, a0l);
            par ^= 1;
        } else if (zh > rs::kZTol && tr.iv == nint - 1) {
            cur = S > 0 ? k1 : k0 - 1;                         // beyond delta, and the rest farther
            break;
        }
        cur += S;
    }
}

// The pairs of one side for one target in a chunk where e-vectors would hardly be shared (the
// chunk's interval range holds more than twice as many (source, interval) e-vectors as it has
// pairs, as where springs lie farther apart than the intervals are wide): each pair folds its own
// source's densities on its interval (the same e-vector, bit for bit, as the shared fold) and
// evaluates it, with no interval windows.  Sources k0 .. k1 - 1 of the chunk.
template <int S>
__device__ __forceinline__ void rs_direct(const float4* sMeta, const float2* sSig, const float* ivt, const int* cell,
                                          float cscale, int nint, int iv_dt, const float4* __restrict__ coef,
                                          const int32_t* __restrict__ mr, int nm, int k0, int k1, int lbj, int nbl,
                                          int nbc, float bh, float bl, rs::Track& tr, float& a0h, float& a0l,
                                          float& a1h, float& a1l) {
    for (int k = k0; k < k1; k++) {
        const float4 mt = sMeta[k];
        const int e = __float_as_int(mt.z), lohi = __float_as_int(mt.w);
        const int lo = lohi & 0x7fff, hi = lohi >> 16;
        if (lo > hi || (S < 0 ? e >= lbj : e < lbj)) continue;
        float zh, zl;
        rs::z_of<S>(tr, mt.x, mt.y, zh, zl);
        if (fabsf(zh) > rs::kZTol) rs::walk<S>(ivt, cell, cscale, nint, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt, iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (!(fabsf(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi)) continue;
        rs::EVec ev;
        rs::evec_zero(ev);
        const int m0 = __ldg(mr + 2 * tr.iv), m1 = __ldg(mr + 2 * tr.iv + 1);
        const float4* c = coef + (size_t)tr.iv * nm * 3;
        const int kk = k & (kRsChunk - 1);
#pragma unroll 1
        for (int m = m0; m <= m1; m++) {
            const float2 sg = sSig[m * kRsChunk + kk];
            const float4 c01 = __ldg(c + 3 * m), c23 = __ldg(c + 3 * m + 1), c47 = __ldg(c + 3 * m + 2);
            rs::acc_mac(ev.e0h, ev.e0l, c01.x, c01.y, sg.x, sg.y);
            rs::acc_mac(ev.e1h, ev.e1l, c01.z, c01.w, sg.x, sg.y);
            ev.e2 = rs::fma_(c23.y, sg.x, rs::fma_(c23.x, sg.x, ev.e2));
            ev.e3 = rs::fma_(c23.w, sg.x, rs::fma_(c23.z, sg.x, ev.e3));
            ev.e4 = rs::fma_(c47.x, sg.x, ev.e4);
            ev.e5 = rs::fma_(c47.y, sg.x, ev.e5);
            ev.e6 = rs::fma_(c47.z, sg.x, ev.e6);
            ev.e7 = rs::fma_(c47.w, sg.x, ev.e7);
        }
        if (k & 1) rs::evec_eval_v(ev, zh, zl, a1h, a1l);
        else rs::evec_eval_v(ev, zh, zl, a0h, a0l);
    }
}

// One side of one target in a block whose targets lie farther apart than two window widths (each
// target meets few of the block's sources): the thread walks its own sources nearest first (left:
// e = lb_j - 1, lb_j - 2, ..; right: e = lb_j, lb_j + 1, ..) until they lie beyond delta, with the
// shared path's per-source data (position on the block grid, interval range over the block, the
// walk and the near/far rule) and one e-vector per pair folded from the density ring itself; no
// shared staging, no barriers.
template <int S>
__device__ __forceinline__ void rs_sparse_side(const DevPlan& P, const RangeDev& R, const float* ivt, float cscale,
                                               rs::Grid G, double xa, double span, double xj, int64_t n, int wlo,
                                               int whi, int lbj, int nbl, int nbc, float bh, float bl, rs::Track& tr,
                                               float& a0h, float& a0l, float& a1h, float& a1l) {
    const double reach = R.delta * (1.0 + 8.0 * rs::kRangeMargin);
    const float4* coef = (const float4*)R.coef;
    for (int q = 0;; q++) {
        const int e = S > 0 ? lbj + q : lbj - 1 - q;
        if (S > 0 ? e >= whi : e < wlo) break;
        const double xe = rs_xext(P, e);
        if (!((S > 0 ? xe - xj : xj - xe) < reach)) break;     // the farther ones lie farther still
        const double xr = xe - xa;
        const int lohi = rs::source_range(xr, S < 0, span, R.delta, P.dt, R.bp2, R.cell, cscale, R.nint);
        const int lo = lohi & 0x7fff, hi = lohi >> 16;
        if (lo > hi) continue;
        float h, l;
        rs::grid_split(xr, G, h, l);
        float zh, zl;
        rs::z_of<S>(tr, h, l, zh, zl);
        if (fabsf(zh) > rs::kZTol) rs::walk<S>(ivt, R.cell, cscale, R.nint, bh, bl, h, l, tr, zh, zl);
        if (lohi & 0x8000) rs::near_side<S>(ivt, R.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, h, l, tr, zh, zl);
        if (!(fabsf(zh) <= rs::kZTol && tr.iv >= lo && tr.iv <= hi)) continue;
        const int64_t sp = rs_spring(e, P.M);
        rs::EVec ev;
        rs::evec_zero(ev);
        const int m0 = __ldg(R.mr + 2 * tr.iv), m1 = __ldg(R.mr + 2 * tr.iv + 1);
        const float4* c = coef + (size_t)tr.iv * R.nm * 3;
#pragma unroll 1
        for (int m = m0; m <= m1; m++) {
            const float2 sg = __ldg((const float2*)P.sig2 + (int64_t)ring_slot(n + 1 - m, P.ring) * P.M + sp);
            const float4 c01 = __ldg(c + 3 * m), c23 = __ldg(c + 3 * m + 1), c47 = __ldg(c + 3 * m + 2);
            rs::acc_mac(ev.e0h, ev.e0l, c01.x, c01.y, sg.x, sg.y);
            rs::acc_mac(ev.e1h, ev.e1l, c01.z, c01.w, sg.x, sg.y);
            ev.e2 = rs::fma_(c23.y, sg.x, rs::fma_(c23.x, sg.x, ev.e2));
            ev.e3 = rs::fma_(c23.w, sg.x, rs::fma_(c23.z, sg.x, ev.e3));
            ev.e4 = rs::fma_(c47.x, sg.x, ev.e4);
            ev.e5 = rs::fma_(c47.y, sg.x, ev.e5);
            ev.e6 = rs::fma_(c47.z, sg.x, ev.e6);
            ev.e7 = rs::fma_(c47.w, sg.x, ev.e7);
        }
        if (q & 1) rs::evec_eval_v(ev, zh, zl, a1h, a1l);
        else rs::evec_eval_v(ev, zh, zl, a0h, a0l);
    }
}

__global__ void __launch_bounds__(kRsTargets, 3) k_rs_local(DevPlan P, RangeDev R) {
    extern __shared__ __align__(16) float rs_sm[];
    float* sE = rs_sm;
    float2* sSig = (float2*)(sE + kRsIvCap * kRsRow);
    float* sIv = (float*)(sSig + (size_t)R.nm * kRsChunk);
    // per source of a group of kRsTargets sources (8 chunks): (h, l, extended index, packed
    // interval range), and the interval union of each chunk
    __shared__ float4 sMeta[kRsTargets];
    __shared__ int sU[2][kRsTargets / kRsChunk];
    // targets' positions relative to the first (float, sorted), and per chunk an estimate of its
    // pairs (sources' targets within delta) for the choice between shared and per-pair e-vectors
    __shared__ float sT[kRsTargets];
    __shared__ int sP[kRsTargets / kRsChunk];

    const int64_t M = P.M;
    const int64_t n = load_step(P);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int64_t j0 = (int64_t)b * kRsTargets;
    const int nT = (int)min((int64_t)kRsTargets, M - j0);
    const double xa = P.x[j0], span = P.x[j0 + nT - 1] - xa;
    const rs::Grid G = rs::grid_of(span, R.delta);
    for (int iv = t; iv < R.nint; iv += blockDim.x) rs::interval_on_grid(__ldg(R.mid + iv), __ldg(R.ih + iv), G, sIv + 4 * iv);
    const float cscale = R.cell_scale;

    const bool valid = t < nT;
    const int64_t j = j0 + (valid ? t : 0);
    const double xj = P.x[j];
    float hj, lj;
    rs::grid_split(xj - xa, G, hj, lj);
    // lb_j: the first spring at x_j's position (sources below it are strictly left of x_j)
    int64_t lbj = j;
    if (j > 0 && P.x[j - 1] == xj) {
        int64_t lo = 0;
        while (lo < lbj) {
            const int64_t mid = (lo + lbj) >> 1;
            if (P.x[mid] < xj) lo = mid + 1;
            else lbj = mid;
        }
    }
    sT[t] = valid ? (float)(xj - xa) : 3.0e38f;
    const int nbl = __ldg(R.nb_lo + j), nbc = __ldg(R.nb_cnt + j);
    const int wlo = __ldg(R.blk_win + 4 * b), inlo = __ldg(R.blk_win + 4 * b + 1);
    const int inhi = __ldg(R.blk_win + 4 * b + 2), whi = __ldg(R.blk_win + 4 * b + 3);
    const int nL = max(0, inhi - wlo), total = nL + max(0, whi - inlo);
    __syncthreads();

    // two accumulators (even and odd sources), so consecutive pairs are independent chains
    float a0h = 0.f, a0l = 0.f, a1h = 0.f, a1l = 0.f;
    rs::Track trL, trR;
    rs::track_to(sIv, 0, hj, lj, trL);
    rs::track_to(sIv, 0, -hj, -lj, trR);

    if (span > 2.0 * R.delta) {
        // targets farther apart than two window widths: no shared e-vectors to speak of
        if (valid) {
            rs_sparse_side<-1>(P, R, sIv, cscale, G, xa, span, xj, n, wlo, whi, (int)lbj, nbl, nbc, hj, lj, trL, a0h, a0l,
                               a1h, a1l);
            rs_sparse_side<1>(P, R, sIv, cscale, G, xa, span, xj, n, wlo, whi, (int)lbj, nbl, nbc, -hj, -lj, trR, a0h,
                              a0l, a1h, a1l);
            P.clocal[j] = ((double)a0h + (double)a0l) + ((double)a1h + (double)a1l);
        }
        return;
    }
    for (int base = 0; base < total; base += kRsChunk) {
        const int grp = base & (kRsTargets - 1);       // the chunk's place in its group of 8
        if (grp == 0) {
            // set-up of the group's 256 sources, one per thread: position on the block grid and
            // interval range; warp w reduces the union of chunk w
            if (base > 0) __syncthreads();             // the previous group's last chunk is done
            const int v = base + t;
            int lohi = 1, e = 0, cnt = 0;
            float h = 0.f, l = 0.f;
            if (v < total) {
                const bool left = v < nL;
                e = left ? wlo + v : inlo + (v - nL);
                const double xr = rs_xext(P, e) - xa;
                rs::grid_split(xr, G, h, l);
                lohi = rs::source_range(xr, left, span, R.delta, P.dt, R.bp2, R.cell, cscale, R.nint);
                if ((lohi & 0x7fff) <= (lohi >> 16)) {
                    // targets within delta of the source (an estimate: float positions)
                    const float xf = (float)xr, df = (float)R.delta;
                    int a = 0, bnd = nT;
                    while (a < bnd) {
                        const int mid = (a + bnd) >> 1;
                        if (sT[mid] > xf - df) bnd = mid;
                        else a = mid + 1;
                    }
                    int c = a;
                    bnd = nT;
                    while (c < bnd) {
                        const int mid = (c + bnd) >> 1;
                        if (sT[mid] >= xf + df) bnd = mid;
                        else c = mid + 1;
                    }
                    cnt = c - a;
                }
            }
            sMeta[t] = make_float4(h, l, __int_as_float(e), __int_as_float(lohi));
            const int lo = lohi & 0x7fff, hi = lohi >> 16;
            int u0 = lo <= hi ? lo : 0x7fffffff, u1 = lo <= hi ? hi : -1;
            for (int o = 16; o > 0; o >>= 1) {
                u0 = min(u0, __shfl_xor_sync(0xffffffffu, u0, o));
                u1 = max(u1, __shfl_xor_sync(0xffffffffu, u1, o));
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            if (lane == 0) {
                sU[0][warp] = u0;
                sU[1][warp] = u1;
                sP[warp] = cnt;
            }
        }
        // the chunk's densities, sigma^{n+1-m} of source k at sSig[m][k] (pairs)
        for (int i = t; i < (R.nm - 1) * kRsChunk; i += blockDim.x) {
            const int k = i & (kRsChunk - 1), m = 1 + i / kRsChunk, v = base + k;
            float2 s = make_float2(0.f, 0.f);
            if (v < total) {
                const int64_t l = rs_spring(v < nL ? wlo + v : inlo + (v - nL), M);
                s = __ldg((const float2*)P.sig2 + (int64_t)ring_slot(n + 1 - m, P.ring) * M + l);
            }
            sSig[m * kRsChunk + k] = s;
        }
        __syncthreads();
        const float4* meta = sMeta + grp;
        const int U0 = sU[0][grp / kRsChunk], U1 = sU[1][grp / kRsChunk];
        if (U1 >= U0 && 2 * sP[grp / kRsChunk] < kRsChunk * (U1 - U0 + 1)) {
            // few pairs per e-vector: each pair folds its own (no windows, no shared records)
            if (valid) {
                const int kend = min(kRsChunk, total - base), kL = min(kend, max(0, nL - base));
                const float4* cf = (const float4*)R.coef;
                rs_direct<-1>(meta, sSig, sIv, R.cell, cscale, R.nint, R.iv_dt, cf, R.mr, R.nm, 0, kL, (int)lbj, nbl, nbc,
                              hj, lj, trL, a0h, a0l, a1h, a1l);
                rs_direct<1>(meta, sSig, sIv, R.cell, cscale, R.nint, R.iv_dt, cf, R.mr, R.nm, kL, kend, (int)lbj, nbl,
                             nbc, -hj, -lj, trR, a0h, a0l, a1h, a1l);
            }
            __syncthreads();
            continue;
        }
        const int lohi_lane = __float_as_int(meta[lane].w);
        const int lo_lane = lohi_lane & 0x7fff, hi_lane = lohi_lane >> 16;
        const bool multi = U1 - U0 + 1 > kRsIvCap;
        const int kend_c = min(kRsChunk, total - base), kL_c = min(kend_c, max(0, nL - base));
        int curL = kL_c - 1, curR = kL_c, par = 0;
        for (int W0 = U0; W0 <= U1; W0 += kRsIvCap) {
            const int W1 = min(U1, W0 + kRsIvCap - 1);
            // e-vectors of the intervals [W0, W1]: warp per interval, lane per source
            for (int iv = W0 + warp; iv <= W1; iv += nwarps) {
                const bool act = lo_lane <= iv && iv <= hi_lane;
                if (!__any_sync(0xffffffffu, act)) continue;
                rs::EVec ev;
                rs::evec_zero(ev);
                const int m0 = __ldg(R.mr + 2 * iv), m1 = __ldg(R.mr + 2 * iv + 1);
                const float4* c = (const float4*)R.coef + (size_t)iv * R.nm * 3;
                // two m per iteration: six coefficient loads in flight (they come from L2)
                int m = m0;
                for (; m < m1; m += 2) {
                    const float4 c01 = __ldg(c + 3 * m), c23 = __ldg(c + 3 * m + 1), c47 = __ldg(c + 3 * m + 2);
                    const float4 d01 = __ldg(c + 3 * m + 3), d23 = __ldg(c + 3 * m + 4), d47 = __ldg(c + 3 * m + 5);
                    const float2 s = sSig[m * kRsChunk + lane], s2 = sSig[(m + 1) * kRsChunk + lane];
                    const float a01[4] = {c01.x, c01.y, c01.z, c01.w}, a23[4] = {c23.x, c23.y, c23.z, c23.w},
                                a47[4] = {c47.x, c47.y, c47.z, c47.w};
                    rs::evec_mac(ev, a01, a23, a47, s.x, s.y);
                    const float b01[4] = {d01.x, d01.y, d01.z, d01.w}, b23[4] = {d23.x, d23.y, d23.z, d23.w},
                                b47[4] = {d47.x, d47.y, d47.z, d47.w};
                    rs::evec_mac(ev, b01, b23, b47, s2.x, s2.y);
                }
                if (m == m1) {
                    const float4 c01 = __ldg(c + 3 * m), c23 = __ldg(c + 3 * m + 1), c47 = __ldg(c + 3 * m + 2);
                    const float2 s = sSig[m * kRsChunk + lane];
                    const float a01[4] = {c01.x, c01.y, c01.z, c01.w}, a23[4] = {c23.x, c23.y, c23.z, c23.w},
                                a47[4] = {c47.x, c47.y, c47.z, c47.w};
                    rs::evec_mac(ev, a01, a23, a47, s.x, s.y);
                }
                float4* rec = (float4*)(sE + (iv - W0) * kRsRow + lane * rs::kERecord);
                rec[0] = make_float4(ev.e0h, ev.e0l, ev.e1h, ev.e1l);
                rec[1] = make_float4(ev.e2, ev.e3, ev.e4, ev.e5);
                rec[2] = make_float4(ev.e6, ev.e7, 0.f, 0.f);
            }
            __syncthreads();
            if (valid && multi) {
                rs_pairs_cursor<-1>(sE, meta, sIv, R.cell, cscale, R.nint, R.iv_dt, 0, kL_c, curL, W0, W1, (int)lbj, nbl,
                                    nbc, hj, lj, trL, par, a0h, a0l, a1h, a1l);
                rs_pairs_cursor<1>(sE, meta, sIv, R.cell, cscale, R.nint, R.iv_dt, kL_c, kend_c, curR, W0, W1, (int)lbj,
                                   nbl, nbc, -hj, -lj, trR, par, a0h, a0l, a1h, a1l);
            } else if (valid) {
                rs_pairs<-1>(sE, meta, sIv, R.cell, cscale, R.nint, R.iv_dt, 0, kL_c, W0, W1, (int)lbj, nbl, nbc, hj, lj,
                             trL, a0h, a0l, a1h, a1l);
                rs_pairs<1>(sE, meta, sIv, R.cell, cscale, R.nint, R.iv_dt, kL_c, kend_c, W0, W1, (int)lbj, nbl, nbc, -hj,
                            -lj, trR, a0h, a0l, a1h, a1l);
            }
            __syncthreads();
        }
    }
    if (valid) P.clocal[j] = ((double)a0h + (double)a0l) + ((double)a1h + (double)a1l);
}

// plan time: the terms of the local sum, sum over pairs (j, l) closer than delta of the number of
// m >= 1 with a non-zero weight on the pair's interval (the multiply-adds sum_m Q_m sigma_l^{n+1-m}
// the method performs per step), by a walk over each target's sources on both sides
__global__ void k_rs_count_terms(DevPlan P, RangeDev R, unsigned long long* total) {
    unsigned long long acc = 0;
    const bool per = P.bc == WAVE1D_PERIODIC;
    const int64_t elo = per ? -P.M : 0, ehi = per ? 2 * P.M : P.M;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x) {
        const double xj = P.x[j];
        for (int side = 0; side < 2; side++) {
            int64_t e = side ? j : j - 1;                  // right: the spring itself first (d = 0)
            int iv = 0;
            for (;;) {
                if (side ? e >= min(ehi, j + P.M) : e < max(elo, j - P.M)) break;
                const double d = side ? rs_xext(P, e) - xj : xj - rs_xext(P, e);
                if (!(d < R.delta)) break;
                while (iv + 1 < R.nint && !(d < __ldg(R.bp + iv + 1))) iv++;
                const int m0 = __ldg(R.mr + 2 * iv), m1 = __ldg(R.mr + 2 * iv + 1);
                acc += (unsigned long long)max(0, m1 - m0 + 1);
                e += side ? 1 : -1;
            }
        }
    }
    atomicAdd(total, acc);
}

// ---------------------------------------------------------------------------------------------
// Implicit solve of eq. linearSystem: (I + S) sigma^{n+1} = rhs by Jacobi sweeps
// ---------------------------------------------------------------------------------------------

// plan time: S_jl = (beta_j / 2) Q_0(d_jl) for the sources of spring j's window (warp per spring)
__global__ void k_rs_nearby_weights(DevPlan P, RangeDev R) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < P.M; j += nw) {
        const double xj = P.x[j], hb = 0.5 * P.beta[j];
        const int lo = R.nb_lo[j], cnt = R.nb_cnt[j];
        const int64_t off = R.nb_off[j];
        for (int k = lane; k < cnt; k += 32) {
            const int64_t e = (int64_t)lo + k;
            const double w = e == j ? 0.0 : hb * rs_q0(R, fabs(rs_xext(P, e) - xj));
            const rs::Pair pw = rs::split(w);
            R.nb_w[2 * (off + k)] = pw.hi;
            R.nb_w[2 * (off + k) + 1] = pw.lo;
        }
        if (lane == 0) R.diag[j] = 1.0 + hb * rs_q0(R, 0.0);
    }
}

__device__ __forceinline__ double rs_from_bits(unsigned long long v) { return __longlong_as_double((long long)v); }

// right-hand side and first iterate: sigma^{n+1} extrapolated from sigma^{n-7..n} (the
// degree-7 polynomial through them), or rhs / (1 + S_jj) in the first steps
__global__ void k_rs_solve_init(DevPlan P, RangeDev R) {
    const int64_t n = load_step(P);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 2 * (kRsMaxIter + 1); i += blockDim.x) R.stats[i] = 0ull;
    const double ex[8] = {8.0, -28.0, 56.0, -70.0, 56.0, -28.0, 8.0, -1.0};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x) {
        const double rhs = fma(-0.5 * P.beta[j], P.clocal[j], __ldcg(P.rhs + j));
        P.rhs[j] = rhs;
        double x0;
        if (n >= 8) {
            x0 = 0.0;
            for (int q = 0; q < 8; q++) x0 = fma(ex[q], P.sig[(int64_t)ring_slot(n - q, P.ring) * P.M + j], x0);
        } else {
            x0 = rhs / R.diag[j];
        }
        R.it64[0][j] = x0;
        const rs::Pair p2 = rs::split(x0);
        R.it2[0][2 * j] = p2.hi;
        R.it2[0][2 * j + 1] = p2.lo;
    }
}

// sweep `it` (1 .. kRsMaxIter): iterate it from iterate it - 1, unless sweep it - 1 converged.
// Warp per spring; the row sum sum_{l != j} S_jl sigma_l in compensated pairs.
__global__ void __launch_bounds__(256) k_rs_jacobi(DevPlan P, RangeDev R, int it) {
    if (it >= 2) {
        const double dmax = rs_from_bits(__ldcg(R.stats + 2 * (it - 1)));
        const double smax = rs_from_bits(__ldcg(R.stats + 2 * (it - 1) + 1));
        if (dmax <= kRsTol * smax) return;
    }
    __shared__ double red[2][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float* src2 = R.it2[(it - 1) & 1];
    const double* src = R.it64[(it - 1) & 1];
    double* dst = R.it64[it & 1];
    float* dst2 = R.it2[it & 1];
    double dmax = 0.0, smax = 0.0;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < P.M; j += nw) {
        const int lo = __ldg(R.nb_lo + j), cnt = __ldg(R.nb_cnt + j);
        const int64_t off = __ldg(R.nb_off + j);
        // four entries per lane in flight (their weight and iterate loads issued together), two
        // accumulators; the row's entries are streamed once per sweep
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
        int k = lane;
        for (; k + 96 < cnt; k += 128) {
            float2 w[4], sv[4];
#pragma unroll
            for (int u = 0; u < 4; u++) w[u] = __ldcs((const float2*)R.nb_w + off + k + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; u++) sv[u] = __ldcg((const float2*)src2 + rs_spring((int64_t)lo + k + 32 * u, P.M));
            rs::acc_mac(ah, al, w[0].x, w[0].y, sv[0].x, sv[0].y);
            rs::acc_mac(bh, bl, w[1].x, w[1].y, sv[1].x, sv[1].y);
            rs::acc_mac(ah, al, w[2].x, w[2].y, sv[2].x, sv[2].y);
            rs::acc_mac(bh, bl, w[3].x, w[3].y, sv[3].x, sv[3].y);
        }
        for (; k < cnt; k += 32) {
            const float2 w = __ldcs((const float2*)R.nb_w + off + k);
            const float2 s = __ldcg((const float2*)src2 + rs_spring((int64_t)lo + k, P.M));
            rs::acc_mac(ah, al, w.x, w.y, s.x, s.y);
        }
        rs::acc_add(ah, al, bh, bl);
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, ah, o), ol = __shfl_xor_sync(0xffffffffu, al, o);
            rs::acc_add(ah, al, oh, ol);
        }
        if (lane == 0) {
            const double x = (__ldcg(P.rhs + j) - ((double)ah + (double)al)) / R.diag[j];
            dmax = fmax(dmax, fabs(x - __ldcg(src + j)));
            smax = fmax(smax, fabs(x));
            dst[j] = x;
            const rs::Pair p2 = rs::split(x);
            dst2[2 * j] = p2.hi;
            dst2[2 * j + 1] = p2.lo;
        }
    }
    if (lane == 0) {
        red[0][wid] = dmax;
        red[1][wid] = smax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            dmax = fmax(dmax, red[0][w]);
            smax = fmax(smax, red[1][w]);
        }
        // non-negative doubles order as their bit patterns (a NaN sorts above every number)
        atomicMax(R.stats + 2 * it, (unsigned long long)__double_as_longlong(dmax));
        atomicMax(R.stats + 2 * it + 1, (unsigned long long)__double_as_longlong(smax));
    }
}

// the converged iterate into the rings: the first sweep whose record meets the stopping rule
// (sweeps after it did not run and left zero records)
__global__ void k_rs_store(DevPlan P, RangeDev R) {
    const int64_t n = load_step(P);
    int fin = kRsMaxIter;
    bool ok = false;
    for (int it = 1; it <= kRsMaxIter; it++) {
        const double dmax = rs_from_bits(__ldcg(R.stats + 2 * it)), smax = rs_from_bits(__ldcg(R.stats + 2 * it + 1));
        if (dmax <= kRsTol * smax) {
            fin = it;
            ok = true;
            break;
        }
    }
    const double* x = R.it64[fin & 1];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x)
        store_sigma(P, n, (int)j, __ldcg(x + j));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *R.iters = fin;
        if (!ok) atomicCAS(P.status, 0, (int)WAVE1D_ENOTCONV);
    }
}

// receivers' local part (eq. localSol2), block (chunk c of 256 sources, receiver r): every m of
// the pair's interval, m = 0 with sigma^{n+1} (already stored), FP64; block sums in a fixed order
__global__ void __launch_bounds__(256) k_rs_receivers(DevPlan P, RangeDev R) {
    __shared__ double red[8];
    const int64_t n = load_step(P);
    const int r = blockIdx.y, c = blockIdx.x;
    const int lo = R.r_win[2 * r], hi = R.r_win[2 * r + 1];
    const int64_t e = (int64_t)lo + (int64_t)c * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (e < hi) {
        const int64_t l = rs_spring(e, P.M);
        const double d = fabs(rs_xext(P, e) - P.xr[r]);
        if (d < R.delta) {
            const int iv = rs_locate64(R, d);
            const double z = (d - __ldg(R.mid + iv)) * (double)__ldg(R.ih + iv);
            const int m0 = __ldg(R.mr0 + 2 * iv), m1 = __ldg(R.mr0 + 2 * iv + 1);
            for (int m = m0; m <= m1; m++) {
                const double q = rs_cheb(R.cheb + ((size_t)iv * R.nm + m) * 8, z);
                v = fma(q, __ldcg(P.sig + (int64_t)ring_slot(n + 1 - m, P.ring) * P.M + l), v);
            }
        }
    }
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        R.r_part[(size_t)r * R.rchunks + c] = s;
    }
}

// u = u_L + u_H at the receivers (chunk partials in order), then the step counter
__global__ void k_rs_finish(DevPlan P, RangeDev R) {
    const int64_t n = load_step(P);
    for (int64_t r = threadIdx.x; r < P.R; r += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < R.rchunks; c++) s += __ldcg(R.r_part + r * R.rchunks + c);
        P.rec_hist[(n % P.chunk) * P.R + r] = 0.5 * s + __ldcg(P.uHr + r);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *P.item_ctr = 0ull;
        P.step[1] = 0;
        __threadfence();
        P.step[0] = n + 1;
    }
}

// ---------------------------------------------------------------------------------------------
// Reverse march (wave1d_adjoint on a plan without pair lists): the transposed local sum,
//   sigmabar_l^{n+1-m} += sum_j Q_m(d_jl) cbar_j,   m >= 1,
// over the same pairs as k_rs_local (every j within delta of l, each once).  On interval iv,
// Q_m(d) = sum_r a_{iv,m,r} z^r, so the pairs of output l that fall in iv enter only through the
// moments F_r = sum_{j in iv} z_jl^r cbar_j, and the interval adds sum_r a_{iv,m,r} F_r to
// output m.  One block of kRsTTargets outputs (thread t: output j0 + t) walks the inputs of its
// window as k_rs_local walks its sources (the same grid, index side test, interval walk and
// near/far rule); a thread accumulates the moments of its current interval (F_0, F_1 as
// compensated pairs, F_2 .. F_7 single) and flushes them into its per-m FP64 outputs in shared
// memory when the interval changes.  No atomics: every output has one writer, in a fixed order.
// ---------------------------------------------------------------------------------------------
size_t rs_local_T_smem(int nint, int nm) {
    return (size_t)4 * nint * sizeof(float) + (size_t)kRsTTargets * nm * sizeof(double) +
           (size_t)kRsChunk * sizeof(float2);
}

struct RsMoments {
    float f0h, f0l, f1h, f1l, f2, f3, f4, f5, f6, f7;
};

// out[m] += sum_r a_{iv,m,r} F_r for the interval's m >= 1 (out: this thread's column, stride kRsTTargets)
__device__ __forceinline__ void rs_flush(const RangeDev& R, int iv, const RsMoments& F, double* out) {
    const int m0 = max(1, __ldg(R.mr + 2 * iv)), m1 = __ldg(R.mr + 2 * iv + 1);
    const float4* c = (const float4*)R.coef + (size_t)iv * R.nm * 3;
    for (int m = m0; m <= m1; m++) {
        const float4 c01 = __ldg(c + 3 * m), c23 = __ldg(c + 3 * m + 1), c47 = __ldg(c + 3 * m + 2);
        float h = 0.f, l = 0.f;
        rs::acc_mac(h, l, c01.x, c01.y, F.f0h, F.f0l);
        rs::acc_mac(h, l, c01.z, c01.w, F.f1h, F.f1l);
        float r = __fmaf_rn(c23.y, F.f2, __fmaf_rn(c23.x, F.f2, 0.f));
        r = __fmaf_rn(c23.w, F.f3, __fmaf_rn(c23.z, F.f3, r));
        r = __fmaf_rn(c47.x, F.f4, r);
        r = __fmaf_rn(c47.y, F.f5, r);
        r = __fmaf_rn(c47.z, F.f6, r);
        r = __fmaf_rn(c47.w, F.f7, r);
        rs::acc_add(h, l, r, 0.f);
        out[(size_t)m * kRsTTargets] += (double)h + (double)l;
    }
}

// F += cbar z^r for one pair (z = zh + zl normalised, cbar = (ch, cl))
__device__ __forceinline__ void rs_moments_add(RsMoments& F, float zh, float zl, float ch, float cl) {
    rs::acc_add(F.f0h, F.f0l, ch, cl);
    rs::acc_mac(F.f1h, F.f1l, zh, zl, ch, cl);
    const float z2 = __fmul_rn(zh, zh);
    float p = __fmul_rn(z2, ch);
    F.f2 = __fadd_rn(F.f2, p);
    p = __fmul_rn(p, zh);
    F.f3 = __fadd_rn(F.f3, p);
    p = __fmul_rn(p, zh);
    F.f4 = __fadd_rn(F.f4, p);
    p = __fmul_rn(p, zh);
    F.f5 = __fadd_rn(F.f5, p);
    p = __fmul_rn(p, zh);
    F.f6 = __fadd_rn(F.f6, p);
    p = __fmul_rn(p, zh);
    F.f7 = __fadd_rn(F.f7, p);
}

// the pairs of one side for one output, inputs [k0, k1) of the chunk (cf. rs_pairs)
template <int S>
__device__ __forceinline__ void rs_pairs_T(const RangeDev& R, const float4* sMeta, const float2* sC, const float* ivt,
                                           float cscale, int k0, int k1, int lbj, int nbl, int nbc, float bh, float bl,
                                           rs::Track& tr, int& cur, RsMoments& F, double* out) {
    for (int kk = k0; kk < k1; kk++) {
        const float4 mt = sMeta[kk];
        const int e = __float_as_int(mt.z), lohi = __float_as_int(mt.w);
        if ((lohi & 0x7fff) > (lohi >> 16) || (S < 0 ? e >= lbj : e < lbj)) continue;
        float zh, zl;
        rs::z_of<S>(tr, mt.x, mt.y, zh, zl);
        if (fabsf(zh) > rs::kZTol) rs::walk<S>(ivt, R.cell, cscale, R.nint, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (lohi & 0x8000)
            rs::near_side<S>(ivt, R.iv_dt, (unsigned)(e - nbl) < (unsigned)nbc, bh, bl, mt.x, mt.y, tr, zh, zl);
        if (!(fabsf(zh) <= rs::kZTol)) continue;
        if (tr.iv != cur) {
            if (cur >= 0) rs_flush(R, cur, F, out);
            cur = tr.iv;
            F = RsMoments{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
        const float2 cb = sC[kk];
        rs_moments_add(F, zh, zl, cb.x, cb.y);
    }
}

__global__ void __launch_bounds__(kRsTTargets) k_rs_local_T(DevPlan P, RangeDev R, int64_t n,
                                                           const double* __restrict__ cbar, double* sb) {
    extern __shared__ __align__(16) float rs_sm[];
    float* sIv = rs_sm;
    double* sOut = (double*)(sIv + 4 * R.nint);                  // [m][thread]
    float2* sC = (float2*)(sOut + (size_t)R.nm * kRsTTargets);   // the chunk's cbar (pairs)
    __shared__ float4 sMeta[kRsTTargets];

    const int64_t M = P.M;
    const int t = threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.x * kRsTTargets;
    const int nT = (int)min((int64_t)kRsTTargets, M - j0);
    const int b = (int)(j0 / kRsTargets);                        // the forward block holding these outputs
    const double xa = P.x[j0], span = P.x[j0 + nT - 1] - xa;
    const rs::Grid G = rs::grid_of(span, R.delta);
    for (int iv = t; iv < R.nint; iv += blockDim.x) rs::interval_on_grid(__ldg(R.mid + iv), __ldg(R.ih + iv), G, sIv + 4 * iv);
    double* out = sOut + t;
    for (int m = 0; m < R.nm; m++) out[(size_t)m * kRsTTargets] = 0.0;
    const bool valid = t < nT;
    const int64_t j = j0 + (valid ? t : 0);
    const double xj = P.x[j];
    float hj, lj;
    rs::grid_split(xj - xa, G, hj, lj);
    int64_t lbj = j;
    if (j > 0 && P.x[j - 1] == xj) {
        int64_t lo = 0;
        while (lo < lbj) {
            const int64_t mid = (lo + lbj) >> 1;
            if (P.x[mid] < xj) lo = mid + 1;
            else lbj = mid;
        }
    }
    const int nbl = __ldg(R.nb_lo + j), nbc = __ldg(R.nb_cnt + j);
    // the forward block's window holds every input within delta of these outputs
    const int wlo = __ldg(R.blk_win + 4 * b), inlo = __ldg(R.blk_win + 4 * b + 1);
    const int inhi = __ldg(R.blk_win + 4 * b + 2), whi = __ldg(R.blk_win + 4 * b + 3);
    const int nL = max(0, inhi - wlo), total = nL + max(0, whi - inlo);
    const float cscale = R.cell_scale;
    __syncthreads();
    rs::Track trL, trR;
    rs::track_to(sIv, 0, hj, lj, trL);
    rs::track_to(sIv, 0, -hj, -lj, trR);
    int cur = -1;
    RsMoments F{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int base = 0; base < total; base += kRsChunk) {
        const int grp = base & (kRsTTargets - 1);                // the chunk's place in its group of 4
        if (grp == 0) {
            __syncthreads();
            const int v = base + t;
            int lohi = 1, e = 0;
            float h = 0.f, l = 0.f;
            if (v < total) {
                const bool left = v < nL;
                e = left ? wlo + v : inlo + (v - nL);
                const double xr = rs_xext(P, e) - xa;
                rs::grid_split(xr, G, h, l);
                lohi = rs::source_range(xr, left, span, R.delta, P.dt, R.bp2, R.cell, cscale, R.nint);
            }
            sMeta[t] = make_float4(h, l, __int_as_float(e), __int_as_float(lohi));
        }
        __syncthreads();
        if (t < kRsChunk) {
            const int v = base + t;
            float2 cb = make_float2(0.f, 0.f);
            if (v < total) {
                const double c = cbar[rs_spring(v < nL ? wlo + v : inlo + (v - nL), M)];
                const float hi = (float)c;
                cb = make_float2(hi, (float)(c - (double)hi));
            }
            sC[t] = cb;
        }
        __syncthreads();
        if (valid) {
            const int kend = min(kRsChunk, total - base), kL = min(kend, max(0, nL - base));
            const float4* meta = sMeta + grp;
            rs_pairs_T<-1>(R, meta, sC, sIv, cscale, 0, kL, (int)lbj, nbl, nbc, hj, lj, trL, cur, F, out);
            rs_pairs_T<1>(R, meta, sC, sIv, cscale, kL, kend, (int)lbj, nbl, nbc, -hj, -lj, trR, cur, F, out);
        }
        __syncthreads();
    }
    if (!valid) return;
    if (cur >= 0) rs_flush(R, cur, F, out);
    for (int m = 1; m < R.nm; m++) {
        const double v = out[(size_t)m * kRsTTargets];
        if (v != 0.0) {
            int64_t q = (n + 1 - m) % P.ring;
            if (q < 0) q += P.ring;
            sb[q * M + j] += v;
        }
    }
}

// Transposed implicit solve.  With S_jl = (beta_j / 2) Q_0(d_jl), (I + S)^T rb = b is
// rb = y / beta with (I + S) y = beta b (beta > 0), so the forward Jacobi sweeps solve it on the
// right-hand side beta b.  Set-up: that right-hand side (k_rs_jacobi reads it as P.rhs) and the
// first iterate rhs / (1 + S_jj); b = sigmabar^{n+1}, taken out of its ring slot.
__global__ void k_rs_adj_init(DevPlan P, RangeDev R, double* __restrict__ slot_vals, double* __restrict__ rhs) {
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 2 * (kRsMaxIter + 1); i += blockDim.x) R.stats[i] = 0ull;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x) {
        const double r = P.beta[j] * slot_vals[j];
        slot_vals[j] = 0.0;
        rhs[j] = r;
        const double x0 = r / R.diag[j];
        R.it64[0][j] = x0;
        const rs::Pair p2 = rs::split(x0);
        R.it2[0][2 * j] = p2.hi;
        R.it2[0][2 * j + 1] = p2.lo;
    }
}

// the converged sweep's y (as k_rs_store chooses it), then rb_j = y_j / beta_j and the step's
// gradient terms and adjoints as the block-solve form gives them (k_adj_solve):
//   grad_j += rb_j (sigma_j^{n+1} [+ g_j^{n+1}]) / beta_j,  gbar_j^{n+1} = -rb_j,  cbar_j = -beta_j rb_j / 2,
//   u_Hbar_j = -beta_j rb_j  (sigma_next, gbar_next in caller order; grad, gbar_next may be null)
__global__ void k_rs_adj_post(DevPlan P, RangeDev R, const double* __restrict__ sigma_next,
                              const double* __restrict__ g_next, double* grad, double* __restrict__ gbar_next,
                              double* cbar, double* uHbar) {
    int fin = kRsMaxIter;
    bool ok = false;
    for (int it = 1; it <= kRsMaxIter; it++) {
        const double dmax = rs_from_bits(__ldcg(R.stats + 2 * it)), smax = rs_from_bits(__ldcg(R.stats + 2 * it + 1));
        if (dmax <= kRsTol * smax) {
            fin = it;
            ok = true;
            break;
        }
    }
    const double* y = R.it64[fin & 1];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.M; j += (int64_t)gridDim.x * blockDim.x) {
        const double bj = P.beta[j];
        const double rb = __ldcg(y + j) / bj;
        const int jc = P.perm[j];
        if (grad) grad[j] += rb * (g_next ? sigma_next[jc] + g_next[jc] : sigma_next[jc]) / bj;
        if (gbar_next) gbar_next[jc] = -rb;
        cbar[j] = -0.5 * bj * rb;
        uHbar[j] = -bj * rb;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !ok) atomicCAS(P.status, 0, (int)WAVE1D_ENOTCONV);
}

// Transposed receiver read-out (eq. localSol2, every m including m = 0, FP64): for spring l and
// each receiver r in order, the extended indices of l inside r's window (those of the forward
// read-out), sigmabar_l^{n+1-m} += (1/2) Q_m(d) ubar_r.  One thread per spring, no atomics.
__global__ void k_rs_adj_receivers(DevPlan P, RangeDev R, int64_t n, const double* __restrict__ ubar, double* sb) {
    const int64_t M = P.M;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < M; l += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t r = 0; r < P.R; r++) {
            const int lo = R.r_win[2 * r], hi = R.r_win[2 * r + 1];
            for (int k = -1; k <= 1; k++) {
                const int64_t e = l + k * M;
                if (e < lo || e >= hi) continue;
                const double d = fabs(rs_xext(P, e) - P.xr[r]);
                if (!(d < R.delta)) continue;
                const int iv = rs_locate64(R, d);
                const double z = (d - __ldg(R.mid + iv)) * (double)__ldg(R.ih + iv);
                const int m0 = __ldg(R.mr0 + 2 * iv), m1 = __ldg(R.mr0 + 2 * iv + 1);
                for (int m = m0; m <= m1; m++) {
                    const double q = rs_cheb(R.cheb + ((size_t)iv * R.nm + m) * 8, z);
                    int64_t s = (n + 1 - m) % P.ring;
                    if (s < 0) s += P.ring;
                    sb[s * M + l] += 0.5 * q * ubar[r];
                }
            }
        }
    }
}

}  // namespace wave1d
