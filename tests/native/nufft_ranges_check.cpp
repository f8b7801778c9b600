// Host-side check of the spreading ranges (no GPU).  Input (stdin): n_inst nf w max_cells
// max_points empty_cells threads, then n_inst + 1 offsets, then the points' first cells (sorted
// within each instance).  Checks that the ranges tile every instance's grid once, that each run of
// a range holds exactly the staged points of its cell (halo cells wrapping round the box), that an
// empty range has no point in reach, that the lane count is the largest that serves every cell,
// and that spreading through the ranges (cell l takes tap t of run l + w - 1 - t) equals direct
// spreading for pseudo-random tap values.  Prints "ok <max relative difference>" or the failure.
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.h"
#include "nufft_host.h"

using namespace wave1d;

int main() {
    int n_inst, nf, w, max_cells, max_points, empty_cells, threads;
    if (std::scanf("%d %d %d %d %d %d %d", &n_inst, &nf, &w, &max_cells, &max_points, &empty_cells, &threads) != 7)
        return 2;
    std::vector<int64_t> off(n_inst + 1);
    for (auto& v : off) if (std::scanf("%lld", (long long*)&v) != 1) return 2;
    const int64_t M = off[n_inst];
    std::vector<int32_t> i0(M);
    for (auto& v : i0) if (std::scanf("%d", &v) != 1) return 2;
    std::vector<NuRange> ranges;
    std::vector<int32_t> runs;
    nufft_ranges(i0, off.data(), n_inst, nf, w, max_cells, max_points, empty_cells, threads, ranges, runs);
    // tap values per point, direct spreading
    std::vector<double> val((size_t)M * w), ref((size_t)n_inst * nf, 0.0), got((size_t)n_inst * nf, 0.0);
    unsigned long long s = 0x9E3779B97F4A7C15ull;
    for (auto& v : val) {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        v = (double)(s >> 11) / 9007199254740992.0 - 0.5;
    }
    std::vector<int> inst(M);
    for (int b = 0; b < n_inst; b++)
        for (int64_t q = off[b]; q < off[b + 1]; q++) inst[q] = b;
    for (int64_t q = 0; q < M; q++)
        for (int t = 0; t < w; t++) ref[(size_t)inst[q] * nf + (i0[q] + t) % nf] += val[(size_t)q * w + t];
    std::vector<int> covered((size_t)n_inst * nf, 0);
    for (const NuRange& r : ranges) {
        const int b = r.c0 / nf, c0 = r.c0 % nf, nr = r.nc + w - 1;
        if (r.nc < 1 || c0 + r.nc > nf) { std::printf("range outside its grid\n"); return 1; }
        for (int l = 0; l < r.nc; l++) covered[r.c0 + l]++;
        if ((nr << r.lg) > threads && r.lg > 0) { std::printf("too many lanes\n"); return 1; }
        if (r.lg < 5 && (nr << (r.lg + 1)) <= threads) { std::printf("lanes not maximal\n"); return 1; }
        const int np = r.na + r.nb;
        if (np == 0) {
            for (int64_t q = off[b]; q < off[b + 1]; q++) {
                const int rel = ((i0[q] - (c0 - w + 1)) % nf + nf) % nf;
                if (rel < nr) { std::printf("empty range with a point in reach\n"); return 1; }
            }
            continue;
        }
        std::vector<int64_t> idx;
        for (int k = 0; k < r.na; k++) idx.push_back(r.a0 + k);
        for (int k = 0; k < r.nb; k++) idx.push_back(r.b0 + k);
        const int32_t* rp = &runs[r.roff];
        if (rp[0] != 0 || rp[nr] != np) { std::printf("run table ends\n"); return 1; }
        // run k holds exactly the instance's points of cell c0 - w + 1 + k (mod nf); a point may be
        // staged twice when the range and its halo wrap round a small grid, once per role
        for (int k = 0; k < nr; k++) {
            if (rp[k + 1] < rp[k]) { std::printf("run table decreasing\n"); return 1; }
            const int cell = ((c0 - w + 1 + k) % nf + nf) % nf;
            int64_t in_cell = 0;
            for (int64_t q = off[b]; q < off[b + 1]; q++) in_cell += i0[q] == cell;
            if (in_cell != rp[k + 1] - rp[k]) { std::printf("run %d holds %d points, its cell %lld\n", k, rp[k + 1] - rp[k], (long long)in_cell); return 1; }
            for (int e = rp[k]; e < rp[k + 1]; e++) {
                const int64_t q = idx[e];
                if (q < off[b] || q >= off[b + 1] || i0[q] != cell) { std::printf("run holds a wrong point\n"); return 1; }
            }
        }
        for (int l = 0; l < r.nc; l++) {
            double a = 0.0;
            for (int t = 0; t < w; t++) {
                const int k = l + w - 1 - t;
                for (int e = rp[k]; e < rp[k + 1]; e++) a += val[(size_t)idx[e] * w + t];
            }
            got[r.c0 + l] = a;
        }
    }
    for (size_t g = 0; g < covered.size(); g++)
        if (covered[g] != 1) { std::printf("grid real %zu covered %d times\n", g, covered[g]); return 1; }
    double worst = 0.0, scale = 1e-300;
    for (size_t g = 0; g < ref.size(); g++) {
        worst = std::fmax(worst, std::fabs(got[g] - ref[g]));
        scale = std::fmax(scale, std::fabs(ref[g]));
    }
    std::printf("ok %.3e\n", worst / scale);
    return 0;
}
