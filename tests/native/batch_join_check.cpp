// Host-side check of joined batch tables (no GPU).  Builds each periodic instance's plan, joins them
// (join_instances) and checks, against the instances' own tables:
//   - the local sum of every spring row and receiver row (items, m >= 1) and the receivers' m = 0
//     terms, for a pseudo-random density history, bit for bit;
//   - the block solve of every spring for pseudo-random right-hand sides, bit for bit;
//   - that the packed solve groups and large-block tasks cover every global spring once, with the
//     lane's item range equal to the joined row's, and that perm is a permutation.
// Input: B dt tol p, then per instance: M R, M positions, M stiffnesses, R receiver positions.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "batch_host.h"
#include "internal.h"
#include "wave1d.h"

using namespace wave1d;

static double hist(int64_t m, int64_t j) { return std::sin(0.37 * (double)m + 1.3 * (double)j) + 0.01 * (double)j; }

// row sums of an item table; src is mapped to the history's spring index by src_map
template <class Map>
static std::vector<double> item_sums(const LocalItems& L, int64_t rows, Map src_map) {
    std::vector<double> out(rows, 0.0);
    for (int64_t r = 0; r < rows; r++)
        for (int64_t it = L.item_ptr[r]; it < L.item_ptr[r + 1]; it++)
            for (int lane = 0; lane < 32; lane++)
                for (int t = 0; t < L.len[it]; t++) {
                    const float* e = &L.w[2 * (L.wbase[it] + 64 * (int64_t)(t >> 1) + 2 * lane + (t & 1))];
                    const int64_t m = L.m_first + L.s0[it] + t;
                    out[r] += ((double)e[0] + (double)e[1]) * hist(m, src_map(L.src[it * 32 + lane]));
                }
    return out;
}

int main() {
    int B, p;
    double dt, tol;
    if (std::scanf("%d %lf %lf %d", &B, &dt, &tol, &p) != 4) return 2;
    std::vector<HostPlan> inst(B);
    std::string err;
    for (int b = 0; b < B; b++) {
        long M, R;
        if (std::scanf("%ld %ld", &M, &R) != 2) return 2;
        std::vector<double> x(M), beta(M), xr(R);
        for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
        for (auto& v : beta) if (std::scanf("%lf", &v) != 1) return 2;
        for (auto& v : xr) if (std::scanf("%lf", &v) != 1) return 2;
        int rc = build_host_plan(x.data(), beta.data(), M, WAVE1D_PERIODIC, dt, 100, tol, p, 0.5, 0, 0, 32, 0, 0,
                                 4096, (int64_t)1 << 34, inst[b], err);
        if (rc == 0) rc = build_receivers(inst[b], xr.data(), R, err);
        if (rc) { std::printf("error %d %s\n", rc, err.c_str()); return 1; }
    }
    BatchTables bt;
    if (join_instances(inst, bt, err)) { std::printf("error %s\n", err.c_str()); return 1; }
    const HostPlan& g = bt.g;
    const int64_t M = g.P.M, R = g.P.R;
    // local sums and receiver terms
    std::vector<double> gl = item_sums(g.litems, M, [](int32_t s) { return (int64_t)s; });
    std::vector<double> gr = item_sums(g.ritems, R, [](int32_t s) { return (int64_t)s; });
    for (int b = 0; b < B; b++) {
        const int64_t mo = bt.moff[b], ro = bt.roff[b];
        auto map = [mo](int32_t s) { return (int64_t)s + mo; };
        std::vector<double> il = item_sums(inst[b].litems, inst[b].P.M, map);
        std::vector<double> ir = item_sums(inst[b].ritems, inst[b].P.R, map);
        for (int64_t j = 0; j < inst[b].P.M; j++)
            if (il[j] != gl[mo + j]) { std::printf("local sum differs: instance %d row %ld\n", b, (long)j); return 1; }
        for (int64_t r = 0; r < inst[b].P.R; r++) {
            if (ir[r] != gr[ro + r]) { std::printf("receiver sum differs\n"); return 1; }
            double a = 0.0, c = 0.0;
            for (int64_t e = inst[b].r0_ptr[r]; e < inst[b].r0_ptr[r + 1]; e++) a += inst[b].r0_w[e] * hist(0, inst[b].r0_src[e] + mo);
            for (int64_t e = g.r0_ptr[ro + r]; e < g.r0_ptr[ro + r + 1]; e++) c += g.r0_w[e] * hist(0, g.r0_src[e]);
            if (a != c) { std::printf("receiver m = 0 terms differ\n"); return 1; }
        }
    }
    // block solves
    std::vector<double> rhs(M), gs(M, 0.0);
    for (int64_t j = 0; j < M; j++) rhs[j] = std::cos(0.7 * (double)j) + 0.5;
    auto solve = [](const HostPlan& h, const std::vector<double>& rr, int64_t off, std::vector<double>& out) {
        for (size_t b = 0; b + 1 < h.blk_ptr.size(); b++) {
            const int64_t m0 = h.blk_ptr[b], s = h.blk_ptr[b + 1] - m0;
            const double* inv = &h.inv[h.blk_inv_off[b]];
            for (int64_t i = 0; i < s; i++) {
                double a = 0.0;
                for (int64_t l = 0; l < s; l++) a += inv[l * s + i] * rr[h.blk_members[m0 + l] + off];
                out[h.blk_members[m0 + i] + off] = a;
            }
        }
    };
    solve(g, rhs, 0, gs);
    for (int b = 0; b < B; b++) {
        std::vector<double> is(M, 0.0);
        solve(inst[b], rhs, bt.moff[b], is);
        for (int64_t j = 0; j < inst[b].P.M; j++)
            if (is[bt.moff[b] + j] != gs[bt.moff[b] + j]) { std::printf("block solve differs\n"); return 1; }
    }
    // solve groups cover every spring once, with the joined row's item range
    std::vector<int> hits(M, 0);
    for (size_t e = 0; e < g.sg_j.size(); e++) {
        const int j = g.sg_j[e];
        if (j < 0) continue;
        if (j >= M) { std::printf("group spring out of range\n"); return 1; }
        hits[j]++;
        if (g.sg_ip[e] != g.litems.item_ptr[j] || g.sg_icnt[e] != g.litems.item_ptr[j + 1] - g.litems.item_ptr[j]) {
            std::printf("group item range differs from the row's\n");
            return 1;
        }
    }
    for (size_t t = 0; t < g.big_blk.size(); t++) {
        const int64_t b = g.big_blk[t], m0 = g.blk_ptr[b], s = g.blk_ptr[b + 1] - m0;
        const int r0 = g.big_row0[t];
        const int rows = s > 256 ? (int)s : std::min<int>(32, (int)s - r0);
        for (int i = 0; i < rows; i++) hits[g.blk_members[m0 + r0 + i]]++;
    }
    std::vector<int> seen(M, 0);
    for (int64_t j = 0; j < M; j++) {
        if (hits[j] != 1) { std::printf("spring %ld solved %d times\n", (long)j, hits[j]); return 1; }
        if (g.perm[j] < 0 || g.perm[j] >= M || seen[g.perm[j]]++) { std::printf("perm is not a permutation\n"); return 1; }
    }
    std::printf("ok %ld %ld %zu\n", (long)M, (long)R, g.litems.row.size());
    return 0;
}
