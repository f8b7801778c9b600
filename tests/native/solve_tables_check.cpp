// Host-side check of the implicit-solve tables (no GPU).  Input (stdin): M dt, then M positions
// and M stiffnesses (free space, tol 1e-12, p = 8).  Emulates the index decoding of the solve
// tasks of the step: packed groups (32 lanes; lane meta = first lane of its block | size << 8 |
// row << 16, right-hand sides exchanged between the lanes of a block) and tasks of 32 rows of
// blocks above 32 members (one task for the whole block above 256 members), and checks that every
// spring is solved exactly once and that its value is row i of its block's inverse applied to the
// block members' right-hand sides.  Prints "ok <max relative difference> <largest block>".
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    long M;
    double dt;
    if (std::scanf("%ld %lf", &M, &dt) != 2) return 2;
    std::vector<double> x(M), beta(M);
    for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : beta) if (std::scanf("%lf", &v) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, WAVE1D_FREE, dt, 100, 1e-12, 8, 0.5, 0, 0, 32, 0, 0, 4096,
                             (int64_t)1 << 34, hp, err);
    if (rc) { std::printf("error %d %s\n", rc, err.c_str()); return 1; }
    std::vector<double> rhs(M);
    for (long j = 0; j < M; j++) rhs[j] = std::sin(1.3 * j + 0.7) + 0.1 * j / (double)M;
    // reference: sigma_j = sum_l inv_b[i][l] rhs[member_b[l]] from the block tables
    const int64_t nb = (int64_t)hp.blk_ptr.size() - 1;
    std::vector<double> ref(M, 0.0), got(M, 0.0);
    std::vector<int> blk_of(M, -1), row_of(M, -1), hits(M, 0);
    int64_t largest = 0;
    for (int64_t b = 0; b < nb; b++) {
        const int64_t m0 = hp.blk_ptr[b], s = hp.blk_ptr[b + 1] - m0;
        largest = std::max(largest, s);
        const double* inv = &hp.inv[hp.blk_inv_off[b]];
        for (int64_t i = 0; i < s; i++) {
            const int j = hp.blk_members[m0 + i];
            blk_of[j] = (int)b;
            row_of[j] = (int)i;
            double a = 0.0;
            for (int64_t l = 0; l < s; l++) a += inv[l * s + i] * rhs[hp.blk_members[m0 + l]];
            ref[j] = a;
        }
    }
    // packed groups, decoded as the step kernel decodes them
    const int64_t ng = (int64_t)hp.sg_smax.size();
    for (int64_t g = 0; g < ng; g++) {
        for (int lane = 0; lane < 32; lane++) {
            const int64_t e = g * 32 + lane;
            const int j = hp.sg_j[e];
            if (j < 0) continue;
            const int meta = hp.sg_meta[e];
            const int b0 = meta & 255, s = (meta >> 8) & 255, i = meta >> 16;
            if (s > hp.sg_smax[g] || b0 + s > 32 || i >= s) { std::printf("bad lane meta\n"); return 1; }
            if (blk_of[j] < 0 || row_of[j] != i) { std::printf("lane row is not the member's row\n"); return 1; }
            const double* invT = &hp.inv[hp.sg_off[e]];
            if (hp.sg_off[e] != hp.blk_inv_off[blk_of[j]]) { std::printf("lane inverse offset\n"); return 1; }
            if (hp.sg_beta[e] != hp.beta[j]) { std::printf("lane stiffness\n"); return 1; }
            if (hp.sg_ip[e] != hp.litems.item_ptr[j] ||
                hp.sg_icnt[e] != hp.litems.item_ptr[j + 1] - hp.litems.item_ptr[j]) {
                std::printf("lane item range\n");
                return 1;
            }
            double a = 0.0;
            for (int l = 0; l < s; l++) {
                const int jl = hp.sg_j[g * 32 + b0 + l];        // the lane the shuffle reads from
                if (jl < 0) { std::printf("shuffle source is an empty lane\n"); return 1; }
                a += invT[(int64_t)l * s + i] * rhs[jl];
            }
            got[j] = a;
            hits[j]++;
        }
    }
    // tasks of big blocks
    for (size_t t = 0; t < hp.big_blk.size(); t++) {
        const int64_t b = hp.big_blk[t];
        const int r0 = hp.big_row0[t];
        const int64_t m0 = hp.blk_ptr[b];
        const int s = (int)(hp.blk_ptr[b + 1] - m0);
        const double* invT = &hp.inv[hp.blk_inv_off[b]];
        std::vector<int> rows;
        if (s <= 256) {
            for (int lane = 0; lane < 32; lane++) if (r0 + lane < s) rows.push_back(r0 + lane);
        } else {
            for (int i = 0; i < s; i++) rows.push_back(i);
        }
        for (int i : rows) {
            double a = 0.0;
            for (int l = 0; l < s; l++) a += invT[(int64_t)l * s + i] * rhs[hp.blk_members[m0 + l]];
            const int j = hp.blk_members[m0 + i];
            got[j] = a;
            hits[j]++;
        }
    }
    double worst = 0.0, scale = 1e-300;
    for (long j = 0; j < M; j++) {
        if (hits[j] != 1) { std::printf("spring %ld solved %d times\n", j, hits[j]); return 1; }
        worst = std::fmax(worst, std::fabs(got[j] - ref[j]));
        scale = std::fmax(scale, std::fabs(ref[j]));
    }
    std::printf("ok %.3e %lld\n", worst / scale, (long long)largest);
    return 0;
}
