// Joining the tables of independent instances into one batched plan (see batch_host.h).
#include "batch_host.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "../../include/wave1d.h"

namespace wave1d {

namespace {

// items of every instance, rows and sources moved by the instances' row / spring offsets and
// weights by the weights before them
void join_items(const std::vector<const LocalItems*>& parts, const std::vector<int64_t>& row_off,
                const std::vector<int64_t>& src_off, LocalItems& out) {
    out = LocalItems();
    out.m_first = parts.empty() ? 1 : parts[0]->m_first;
    out.item_ptr.assign(1, 0);
    int64_t items = 0, weights = 0;
    for (size_t b = 0; b < parts.size(); b++) {
        const LocalItems& L = *parts[b];
        const int64_t rows = (int64_t)L.item_ptr.size() - 1;
        for (int64_t r = 0; r < rows; r++) out.item_ptr.push_back(L.item_ptr[r + 1] + items);
        for (int32_t r : L.row) out.row.push_back((int32_t)(r + row_off[b]));
        out.s0.insert(out.s0.end(), L.s0.begin(), L.s0.end());
        out.len.insert(out.len.end(), L.len.begin(), L.len.end());
        const int64_t ni = (int64_t)L.row.size();       // wbase holds ni + 1 entries: the last is the total
        for (int64_t c = 0; c < ni; c++) out.wbase.push_back(L.wbase[c] + weights);
        for (int32_t s : L.src) out.src.push_back((int32_t)(s + src_off[b]));
        out.w.insert(out.w.end(), L.w.begin(), L.w.end());
        items += ni;
        weights += (int64_t)L.w.size() / 2;
    }
    out.wbase.push_back(weights);
}

}  // namespace

int join_instances(const std::vector<HostPlan>& inst, BatchTables& out, std::string& err) {
    const size_t B = inst.size();
    if (B == 0) { err = "no instances"; return WAVE1D_EINVAL; }
    const Params& P0 = inst[0].P;
    for (const HostPlan& h : inst) {
        const Params& P = h.P;
        if (P.K != P0.K || P.W != P0.W || P.m_max != P0.m_max || P.nf != P0.nf || P.L1 != P0.L1 ||
            P.nufft_w != P0.nufft_w || P.p != P0.p || P.ring != P0.ring || P.bc != P0.bc ||
            h.litems.m_first != inst[0].litems.m_first || h.ritems.m_first != inst[0].ritems.m_first) {
            err = "instances with different derived sizes";
            return WAVE1D_EINVAL;
        }
    }
    out = BatchTables();
    HostPlan& g = out.g;
    out.moff.assign(B + 1, 0);
    out.roff.assign(B + 1, 0);
    for (size_t b = 0; b < B; b++) {
        out.moff[b + 1] = out.moff[b] + inst[b].P.M;
        out.roff[b + 1] = out.roff[b] + inst[b].P.R;
    }
    const int64_t M = out.moff[B], R = out.roff[B];
    g.P = P0;
    g.P.M = M;
    g.P.R = R;
    // shared history tables
    g.pq = inst[0].pq;
    g.rot = inst[0].rot;
    g.deconv1 = inst[0].deconv1;
    g.deconv2 = inst[0].deconv2;
    g.twiddle = inst[0].twiddle;
    g.modefac = inst[0].modefac;
    g.tw2K = inst[0].tw2K;
    out.inst_of.assign(M, 0);
    for (size_t b = 0; b < B; b++) {
        const HostPlan& h = inst[b];
        const int64_t mo = out.moff[b];
        for (int64_t j = 0; j < h.P.M; j++) {
            g.x.push_back(h.x[j]);
            g.beta.push_back(h.beta[j]);
            g.perm.push_back((int32_t)(h.perm[j] + mo));
            out.inst_of[mo + j] = (int32_t)b;
        }
        g.xr.insert(g.xr.end(), h.xr.begin(), h.xr.end());
    }
    // local-sum items of the springs (rows: springs) and of the receivers (rows: receivers)
    std::vector<const LocalItems*> lp, rp;
    for (const HostPlan& h : inst) {
        lp.push_back(&h.litems);
        rp.push_back(&h.ritems);
    }
    join_items(lp, out.moff, out.moff, g.litems);
    join_items(rp, out.roff, out.moff, g.ritems);
    // receivers' m = 0 terms
    g.r0_ptr.assign(1, 0);
    for (size_t b = 0; b < B; b++) {
        const HostPlan& h = inst[b];
        const int64_t base = (int64_t)g.r0_src.size();
        for (int64_t r = 0; r < h.P.R; r++) g.r0_ptr.push_back(h.r0_ptr[r + 1] + base);
        for (int32_t s : h.r0_src) g.r0_src.push_back((int32_t)(s + out.moff[b]));
        g.r0_w.insert(g.r0_w.end(), h.r0_w.begin(), h.r0_w.end());
    }
    // blocks of I + S, their inverses and the packed solve groups
    g.blk_ptr.assign(1, 0);
    std::vector<int64_t> item_off(B + 1, 0), blk_off(B + 1, 0);
    for (size_t b = 0; b < B; b++) {
        item_off[b + 1] = item_off[b] + (int64_t)inst[b].litems.row.size();
        blk_off[b + 1] = blk_off[b] + (int64_t)inst[b].blk_ptr.size() - 1;
    }
    for (size_t b = 0; b < B; b++) {
        const HostPlan& h = inst[b];
        const int64_t mo = out.moff[b], io = (int64_t)g.inv.size();
        for (size_t k = 1; k < h.blk_ptr.size(); k++) g.blk_ptr.push_back(h.blk_ptr[k] + mo);
        for (int32_t j : h.blk_members) g.blk_members.push_back((int32_t)(j + mo));
        const int64_t nb = (int64_t)h.blk_ptr.size() - 1;    // blk_inv_off holds nb + 1 entries (last: total)
        for (int64_t k = 0; k < nb; k++) g.blk_inv_off.push_back(h.blk_inv_off[k] + io);
        g.inv.insert(g.inv.end(), h.inv.begin(), h.inv.end());
        for (int32_t j : h.sg_j) g.sg_j.push_back(j >= 0 ? (int32_t)(j + mo) : j);
        g.sg_meta.insert(g.sg_meta.end(), h.sg_meta.begin(), h.sg_meta.end());
        for (int64_t o : h.sg_off) g.sg_off.push_back(o + io);
        g.sg_beta.insert(g.sg_beta.end(), h.sg_beta.begin(), h.sg_beta.end());
        for (int64_t ip : h.sg_ip) g.sg_ip.push_back(ip + item_off[b]);
        g.sg_icnt.insert(g.sg_icnt.end(), h.sg_icnt.begin(), h.sg_icnt.end());
        g.sg_smax.insert(g.sg_smax.end(), h.sg_smax.begin(), h.sg_smax.end());
        for (int64_t k : h.big_blk) g.big_blk.push_back(k + blk_off[b]);
        g.big_row0.insert(g.big_row0.end(), h.big_row0.begin(), h.big_row0.end());
        g.max_block = std::max(g.max_block, h.max_block);
    }
    g.blk_inv_off.push_back((int64_t)g.inv.size());
    return WAVE1D_OK;
}

InstanceShape instance_shape(const double* x, int64_t M, double dt, double delta) {
    InstanceShape out;
    if (M < 1) return out;
    const double two_pi = 2.0 * 3.14159265358979323846;
    std::vector<double> v((size_t)M);
    for (int64_t j = 0; j < M; j++) {
        double a = std::fmod(x[j] + 0.5 * two_pi, two_pi);
        if (a < 0) a += two_pi;
        v[j] = a - 0.5 * two_pi;
    }
    std::sort(v.begin(), v.end());
    // gap g_i between sorted neighbours i and i + 1, the last one across the seam
    auto gap = [&](int64_t i) { return i + 1 < M ? v[i + 1] - v[i] : v[0] + two_pi - v[M - 1]; };
    int64_t start = -1;
    for (int64_t i = 0; i < M && start < 0; i++)
        if (!(gap(i) < dt)) start = i;
    if (start < 0 || M == 1) {
        out.largest_block = M;
    } else {
        // walk the circle from the spring after a break; a run ends at each gap of dt or more
        int64_t run = 1;
        for (int64_t k = 1; k <= M; k++) {
            const int64_t i = (start + k) % M;
            out.largest_block = std::max(out.largest_block, run);
            run = gap(i) < dt ? run + 1 : 1;
        }
    }
    // sources l != j within delta of j: the sorted circle doubled, each unordered pair once
    int64_t hi = 0, pairs = 0;
    for (int64_t j = 0; j < M; j++) {
        if (hi < j + 1) hi = j + 1;
        auto pos = [&](int64_t e) { return e < M ? v[e] : v[e - M] + two_pi; };
        while (hi < j + M && pos(hi) - v[j] < delta) hi++;
        pairs += hi - (j + 1);
    }
    out.pairs = 2 * pairs;
    return out;
}

int batch_instances(int n_inst, const int64_t* offsets, const double* x, const double* beta,
                    const int64_t* r_offsets, const double* xr, double dt, int64_t Nt, double tol,
                    const wave1d_opts& o, std::vector<int>& form, std::vector<int>& joined,
                    std::vector<HostPlan>& inst, std::string& err) {
    auto R_of = [&](int b) { return r_offsets ? r_offsets[b + 1] - r_offsets[b] : (int64_t)0; };
    form.assign((size_t)n_inst, o.local_weights == 1 ? 1 : 0);
    if (o.local_weights == 2) {
        const double delta = window_steps(tol, o.gamma, o.W) * dt;
        for (int b = 0; b < n_inst; b++) {
            const InstanceShape sh = instance_shape(x + offsets[b], offsets[b + 1] - offsets[b], dt, delta);
            if (sh.largest_block > o.max_block || sh.pairs > kBatchPairs) form[b] = 1;
        }
    }
    joined.clear();
    inst.clear();
    // The candidates are built side by side in groups whose stored weights, bounded above by
    // (pairs + M) (m_max + 1) doubles each, fit together in what is left of the budget (so none of
    // them can fail it, and their host memory stays within it); a candidate that does not fit
    // alone is built alone against the rest of the budget.  Each group is then taken in instance
    // order with the budget's exact accounting: the same split as one build after another.
    std::vector<int> cand;
    for (int b = 0; b < n_inst; b++)
        if (form[b] == 0) cand.push_back(b);
    const size_t nc = cand.size();
    const double delta = window_steps(tol, o.gamma, o.W) * dt;
    const int m_max = window_steps(tol, o.gamma, o.W) + (o.p + 1) / 2;
    std::vector<double> est(nc);
    for (size_t k = 0; k < nc; k++) {
        const int b = cand[k];
        const int64_t M = offsets[b + 1] - offsets[b];
        const InstanceShape sh = instance_shape(x + offsets[b], M, dt, delta);
        est[k] = ((double)sh.pairs * 1.01 + 2.0 * (double)M + 64.0) * (double)(m_max + 1) * 8.0;
    }
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    int64_t bytes = 0;
    for (size_t k0 = 0; k0 < nc;) {
        const int64_t left = o.max_local_bytes - bytes;
        size_t k1 = k0 + 1;
        for (double sum = est[k0]; sum <= (double)left && k1 < nc && sum + est[k1] <= (double)left; k1++)
            sum += est[k1];
        const size_t ng = k1 - k0;
        std::vector<HostPlan> built(ng);
        std::vector<int> status(ng, WAVE1D_OK);
        std::vector<std::string> why(ng);
        std::atomic<size_t> next{0};
        auto work = [&] {
            for (size_t g = next++; g < ng; g = next++) {
                const int b = cand[k0 + g];
                int rc = build_host_plan(x + offsets[b], beta + offsets[b], offsets[b + 1] - offsets[b],
                                         WAVE1D_PERIODIC, dt, Nt, tol, o.p, o.gamma, o.W, o.NL, o.Ng, 0, o.rbc_period,
                                         o.max_block, left, built[g], why[g]);
                if (rc == WAVE1D_OK) {
                    double none = 0.0;
                    const int64_t R = R_of(b);
                    rc = build_receivers(built[g], R ? xr + r_offsets[b] : &none, R, why[g]);
                }
                status[g] = rc;
            }
        };
        std::vector<std::thread> pool;
        for (size_t t = 1; t < std::min(ng, hw); t++) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
        for (size_t g = 0; g < ng; g++) {
            const int b = cand[k0 + g];
            int rc = status[g];
            if (rc == WAVE1D_OK && (double)built[g].loc.woff.back() * 8.0 > (double)(o.max_local_bytes - bytes)) {
                rc = WAVE1D_ENOMEM;
                why[g] = "local weights need " + std::to_string(built[g].loc.woff.back() * 8) +
                         " bytes, over the budget max_local_bytes";
            }
            if (rc == WAVE1D_ENOMEM && o.local_weights == 2) {
                form[b] = 1;
                continue;
            }
            if (rc) {
                err = "instance " + std::to_string(b) + ": " + why[g];
                return rc;
            }
            bytes += (int64_t)built[g].litems.w.size() * 4;
            inst.push_back(std::move(built[g]));
            joined.push_back(b);
        }
        k0 = k1;
    }
    return WAVE1D_OK;
}

}  // namespace wave1d
