// Host-side check of the reverse-time (adjoint) step (no GPU).  Builds the plan tables for a
// layout read from stdin and runs the bodies the adjoint kernels run (adjoint.cuh) over them, one
// element at a time, in the kernels' launch order; the two transforms of the reverse step are
// exact Fourier sums here (the library uses its NUFFT plan).  Prints "ok", the gradient dL/dbeta
// (caller order) and, for a march driven by forcing vectors, dL/dg (Nt x M, caller order).
// Input: M R bc dt tol p Nt has_g, then M positions, M stiffnesses, R receiver positions, Nt x M
// densities (row s = sigma^{s+1}, caller order), Nt x R receiver adjoints (row s = dL/du^{s+1})
// and, if has_g, Nt x M forcing vectors (row s = g^{s+1}, caller order).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "adjoint_host.h"
#include "internal.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    long M, R, Nt;
    int bc, p, has_g;
    double dt, tol;
    if (std::scanf("%ld %ld %d %lf %lf %d %ld %d", &M, &R, &bc, &dt, &tol, &p, &Nt, &has_g) != 8) return 2;
    std::vector<double> x(M), beta(M), xr(R), sig((size_t)Nt * M), ubar((size_t)Nt * R),
        gin(has_g ? (size_t)Nt * M : 0), gbar(has_g ? (size_t)Nt * M : 0);
    for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : beta) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : xr) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : sig) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : ubar) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : gin) if (std::scanf("%lf", &v) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, bc, dt, Nt, tol, p, 0.5, 0, 0, 32, 0, 0, 4096,
                             (int64_t)1 << 34, hp, err);
    if (rc == 0) rc = build_receivers(hp, xr.data(), R, err);
    if (rc) {
        std::printf("error %d %s\n", rc, err.c_str());
        return 1;
    }
    const Params& P = hp.P;
    const int K = P.K, K1 = K + 1, W = P.W, ring = P.ring;
    // every index the adjoint kernels form stays inside its table
    auto items_in_bounds = [&](const LocalItems& it, int64_t rows) {
        const int64_t n = (int64_t)it.row.size();
        if ((int64_t)it.item_ptr.size() != rows + 1 || it.item_ptr[rows] != n) return false;
        if ((int64_t)it.src.size() != 32 * n) return false;
        for (int64_t o = 0; o < n; o++) {
            if (it.row[o] < 0 || it.row[o] >= rows || it.len[o] < 0) return false;
            if (it.len[o] > 0 && 2 * (it.wbase[o] + 64 * (int64_t)((it.len[o] - 1) >> 1) + 2 * 31 + 1) + 1 >= (int64_t)it.w.size())
                return false;
            if (it.m_first + it.s0[o] < 1 || it.m_first + it.s0[o] + it.len[o] - 1 > P.m_max) return false;
            for (int l = 0; l < 32; l++)
                if (it.src[o * 32 + l] < 0 || it.src[o * 32 + l] >= M) return false;
        }
        return true;
    };
    bool ok = items_in_bounds(hp.litems, M) && items_in_bounds(hp.ritems, R) &&
              (int64_t)hp.pq.size() == 2 * (int64_t)W * K1 && (int64_t)hp.rot.size() == 3 * (int64_t)K1 &&
              (int64_t)hp.tw2K.size() == 4 * (int64_t)K && hp.rbc_phi.size() == hp.rbc_idx.size() &&
              hp.rbc_dphi.size() == hp.rbc_idx.size() && (int64_t)hp.blk_members.size() == M &&
              ring == P.m_max + 1;
    for (int32_t i : hp.rbc_idx) ok = ok && i >= 0 && i < 2 * K;
    for (size_t b = 0; ok && b + 1 < hp.blk_ptr.size(); b++) {
        const int64_t s = hp.blk_ptr[b + 1] - hp.blk_ptr[b];
        ok = s >= 1 && hp.blk_inv_off[b] + s * s <= (int64_t)hp.inv.size();
    }
    for (int64_t e = 0; ok && e < (int64_t)hp.r0_src.size(); e++) ok = hp.r0_src[e] >= 0 && hp.r0_src[e] < M;
    if (!ok) {
        std::printf("index out of bounds\n");
        return 1;
    }
    std::vector<double> sb((size_t)ring * M, 0.0), Sb((size_t)W * K1 * 2, 0.0), ab(2 * K1, 0.0),
        apb(2 * K1, 0.0), a2(2 * K1, 0.0), S1(2 * K1, 0.0), grad(M, 0.0), tmp(M), cbar(M), uHbar(M);
    std::vector<int32_t> blk_of(M);
    const int64_t nb = (int64_t)hp.blk_ptr.size() - 1;
    for (int64_t b = 0; b < nb; b++)
        for (int64_t e = hp.blk_ptr[b]; e < hp.blk_ptr[b + 1]; e++) blk_of[e] = (int32_t)b;
    const int npts = (int)hp.rbc_idx.size();
    std::vector<double> uvbar(2 * (size_t)std::max(npts, 1));
    const double two_pi = 6.283185307179586476925286766559;
    ReceiverColumns rcol;
    receiver_columns(hp.rloc, M, rcol);
    for (size_t e = 0; ok && e < rcol.rcv.size(); e++) {
        const int lo = rcol.mrange[e] & 0xffff, cnt = rcol.mrange[e] >> 16;
        ok = rcol.rcv[e] >= 0 && rcol.rcv[e] < R && lo >= 0 && lo + cnt - 1 <= P.m_max &&
             rcol.woff[e] + cnt <= (int64_t)hp.rloc.w.size();
    }
    if (!ok || (int64_t)rcol.src_ptr.size() != M + 1) {
        std::printf("index out of bounds\n");
        return 1;
    }
    const int nm = P.m_max + 1, stride = 33;
    std::vector<float> acc(2 * (size_t)nm * stride);

    for (int64_t n = Nt - 1; n >= 0; n--) {
        const double* ub = ubar.data() + n * R;
        // receivers: one writer per source, m >= 0
        for (long l = 0; l < M; l++)
            adj::receivers_T_source(l, rcol.src_ptr.data(), rcol.rcv.data(), rcol.mrange.data(), rcol.woff.data(),
                                    hp.rloc.w.data(), ub, n + 1, ring,
                                    [&](int s, double v) { sb[(size_t)s * M + l] += v; });
        // take sigmabar^{n+1}
        double* s1 = sb.data() + (size_t)adj::slot(n + 1, ring) * M;
        for (long j = 0; j < M; j++) { tmp[j] = s1[j]; s1[j] = 0.0; }
        // transposed solve and the gradient term
        for (long e = 0; e < M; e++) {
            const int b = blk_of[e];
            const int64_t m0 = hp.blk_ptr[b];
            const int s = (int)(hp.blk_ptr[b + 1] - m0);
            const double rb = adj::solve_T(hp.inv.data() + hp.blk_inv_off[b], hp.blk_members.data(), m0, s,
                                           (int)(e - m0), tmp.data());
            const int j = hp.blk_members[e];
            const int jc = hp.perm[j];
            const double term = has_g ? sig[(size_t)n * M + jc] + gin[(size_t)n * M + jc] : sig[(size_t)n * M + jc];
            grad[j] += rb * term / hp.beta[j];
            if (has_g) gbar[(size_t)n * M + jc] = -rb;
            cbar[j] = -0.5 * hp.beta[j] * rb;
            uHbar[j] = -hp.beta[j] * rb;
        }
        if (n == 0) break;
        // transposed local sum: row l's items read in the transposed direction, compensated FP32
        // pairs per (m, lane), then FP64 lane sums in lane order
        const LocalItems& li = hp.litems;
        for (long l = 0; l < M; l++) {
            std::fill(acc.begin(), acc.end(), 0.0f);
            for (int64_t it = li.item_ptr[l]; it < li.item_ptr[l + 1]; it++)
                for (int lane = 0; lane < 32; lane++) {
                    float ch, cl;
                    adj::split_pair(cbar[li.src[it * 32 + lane]], ch, cl);
                    adj::item_lane_gather(li.w.data(), li.wbase[it], li.s0[it], li.len[it], lane, li.m_first, ch, cl,
                                          [&](int m) { return &acc[2 * ((size_t)m * stride + lane)]; });
                }
            for (int m = 0; m < nm; m++) {
                double sm = 0.0;
                for (int i = 0; i < 32; i++)
                    sm += (double)acc[2 * ((size_t)m * stride + i)] + (double)acc[2 * ((size_t)m * stride + i) + 1];
                if (sm != 0.0) sb[(size_t)adj::slot(n + 1 - m, ring) * M + l] += sm;
            }
        }
        // type-1 of u_Hbar (exact): S1_k = (1/2 pi) sum_j u_Hbar_j e^{i k x_j}
        for (int k = 0; k <= K; k++) {
            double re = 0.0, im = 0.0;
            for (long j = 0; j < M; j++) {
                re += uHbar[j] * std::cos(k * hp.x[j]);
                im += uHbar[j] * std::sin(k * hp.x[j]);
            }
            S1[2 * k] = re / two_pi;
            S1[2 * k + 1] = im / two_pi;
        }
        for (int k = 0; k <= K; k++) adj::modes_in(k, S1.data(), hp.xr.data(), ub, R, ab.data());
        if (P.bc == WAVE1D_FREE && (n + 1) % P.rbc_period == 0) {
            for (int pt = 0; pt < npts; pt++)
                adj::rbc_grid_T(hp.rbc_idx[pt], K, hp.tw2K.data(), ab.data(), apb.data(), hp.rbc_phi[pt],
                                hp.rbc_dphi[pt], &uvbar[2 * pt], &uvbar[2 * pt + 1]);
            for (int k = 0; k <= K; k++)
                adj::rbc_update_T(k, K, npts, hp.rbc_idx.data(), hp.tw2K.data(), uvbar.data(), ab.data(), apb.data());
        }
        for (int k = 0; k <= K; k++)
            adj::modes_T(k, K1, W, n, hp.rot.data(), hp.pq.data(), ab.data(), apb.data(), Sb.data(), a2.data());
        // type-2 of a2 at the springs (exact), added to sigmabar^n
        double* s0 = sb.data() + (size_t)adj::slot(n, ring) * M;
        for (long j = 0; j < M; j++) {
            double u = a2[0];
            for (int k = 1; k <= K; k++)
                u += 2.0 * (a2[2 * k] * std::cos(k * hp.x[j]) + a2[2 * k + 1] * std::sin(k * hp.x[j]));
            s0[j] += u;
        }
    }
    std::vector<double> out(M);
    for (long j = 0; j < M; j++) out[hp.perm[j]] = grad[j];
    std::printf("ok");
    for (long j = 0; j < M; j++) std::printf(" %.17g", out[j]);
    for (double v : gbar) std::printf(" %.17g", v);
    std::printf("\n");
    return 0;
}
