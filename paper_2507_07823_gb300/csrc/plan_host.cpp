// Host-side plan construction: everything that depends only on the geometry and the
// parameters, computed once before the time march (the paper's "precomputation", Sec. 4.3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <numeric>
#include <thread>

#include "adjoint_host.h"
#include "internal.h"
#include "nufft_host.h"
#include "../../include/wave1d.h"

namespace wave1d {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, n / 256));
    if (nt <= 1) {
        body(0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (int64_t t = 0; t < nt; t++) {
        int64_t a = t * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([=, &body] { body(a, b); });
    }
    for (auto& t : th) t.join();
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& xs, std::vector<double>& ws) {
    xs.assign(n, 0.0);
    ws.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; i++) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // one more update of dp at the converged node
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; k++) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        xs[i] = -z;
        xs[n - 1 - i] = z;
        ws[i] = ws[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) xs[n / 2] = 0.0;
}

double bessel_i0(double z) { return std::cyl_bessel_i(0.0, z); }
double bessel_i1(double z) { return std::cyl_bessel_i(1.0, z); }

// ---------------------------------------------------------------------------------------------
// Blending window of eq. phi: phi' is the Kaiser-Bessel bump scaled to [0, delta]; phi is its
// integral.  phi is tabulated on [0, delta/2] by Chebyshev panels built from Gauss-Legendre
// integrals of phi', and reflected with phi(t) = 1 - phi(delta - t) (phi' is symmetric).
// ---------------------------------------------------------------------------------------------
class Window {
  public:
    Window(double delta, double b) : delta_(delta), b_(b) {
        scale_ = b_ / (delta_ * std::sinh(b_));
        gauss_legendre(40, gx_, gw_);
        double half = 0.5 * delta_;
        pw_ = half / kPanels;
        coef_.assign(kPanels * (kDeg + 1), 0.0);
        double base = 0.0;
        for (int pnl = 0; pnl < kPanels; pnl++) {
            double a = pnl * pw_;
            double vals[kDeg + 1];
            for (int i = 0; i <= kDeg; i++) {
                double c = std::cos(kPi * (i + 0.5) / (kDeg + 1));   // Chebyshev points, 1st kind
                double t = a + 0.5 * pw_ * (c + 1.0);
                vals[i] = base + integral(a, t);
            }
            for (int m = 0; m <= kDeg; m++) {
                double s = 0.0;
                for (int i = 0; i <= kDeg; i++)
                    s += vals[i] * std::cos(kPi * m * (i + 0.5) / (kDeg + 1));
                coef_[pnl * (kDeg + 1) + m] = s * (m == 0 ? 1.0 : 2.0) / (kDeg + 1);
            }
            base += integral(a, a + pw_);
        }
    }
    double delta() const { return delta_; }
    double dphi(double t) const {
        if (t < 0.0 || t > delta_) return 0.0;
        double u = 2.0 * t / delta_ - 1.0;
        double r = 1.0 - u * u;
        return scale_ * bessel_i0(b_ * std::sqrt(r > 0.0 ? r : 0.0));
    }
    // phi''(t) = -(2 b^3 u / (delta^2 sinh b)) I1(z)/z, z = b sqrt(1 - u^2)
    double ddphi(double t) const {
        if (t < 0.0 || t > delta_) return 0.0;
        double u = 2.0 * t / delta_ - 1.0;
        double r = 1.0 - u * u;
        double z = b_ * std::sqrt(r > 0.0 ? r : 0.0);
        double i1z = z > 1e-8 ? bessel_i1(z) / z : 0.5;
        return -(2.0 * b_ * b_ * b_ * u / (delta_ * delta_ * std::sinh(b_))) * i1z;
    }
    double phi(double t) const {
        if (t <= 0.0) return 0.0;
        if (t >= delta_) return 1.0;
        if (t <= 0.5 * delta_) return low(t);
        return 1.0 - low(delta_ - t);
    }

  private:
    static constexpr int kPanels = 48;
    static constexpr int kDeg = 18;
    double integral(double a, double c) const {
        double s = 0.0, hw = 0.5 * (c - a);
        for (size_t i = 0; i < gx_.size(); i++) s += gw_[i] * dphi(a + hw * (gx_[i] + 1.0));
        return s * hw;
    }
    double low(double t) const {
        int pnl = std::min(kPanels - 1, (int)(t / pw_));
        double z = 2.0 * (t - pnl * pw_) / pw_ - 1.0;
        const double* c = &coef_[pnl * (kDeg + 1)];
        double b0 = 0.0, b1 = 0.0;      // Clenshaw
        for (int m = kDeg; m >= 1; m--) {
            double b2 = b1;
            b1 = b0;
            b0 = 2.0 * z * b1 - b2 + c[m];
        }
        return z * b0 - b1 + c[0];
    }
    double delta_, b_, scale_, pw_;
    std::vector<double> gx_, gw_, coef_;
};

// sin(k a)/k with the k = 0 limit a (Remark r:kzero)
inline double sinc_k(double k, double a) { return k == 0.0 ? a : std::sin(k * a) / k; }

// ---------------------------------------------------------------------------------------------
// Local weights Q_m(d), m = 0..m_max (Sec. 4.1): an NL-point Gauss-Legendre rule over the
// look-back interval s in [d, delta] (s = t_{n+1} - tau) of (1 - phi(s)) times the p-point
// interpolant through the nearest available grid times m dt, m_min <= m <= m_max, with
// m_min = 0 for d < dt (nearby, implicit) and 1 otherwise.  Barycentric Lagrange weights.
// ---------------------------------------------------------------------------------------------
struct LocalRule {
    const Params* P;
    const Window* win;
    std::vector<double> gx, gw, lam;       // GL rule; barycentric weights of p equispaced points
    void init(const Params& Pp, const Window& w) {
        P = &Pp;
        win = &w;
        gauss_legendre(Pp.NL, gx, gw);
        lam.assign(Pp.p, 0.0);
        // lambda_r = (-1)^r binom(p-1, r) for equispaced nodes (common factor dropped)
        double c = 1.0;
        for (int r = 0; r < Pp.p; r++) {
            lam[r] = (r % 2 == 0 ? 1.0 : -1.0) * c;
            c = c * (Pp.p - 1 - r) / (r + 1);
        }
    }
    // fills Q[0..m_max]; returns false if every weight is zero (d >= delta)
    bool weights(double d, double* Q) const {
        const Params& p = *P;
        for (int m = 0; m <= p.m_max; m++) Q[m] = 0.0;
        if (!(d < p.delta)) return false;
        int m_min = d < p.dt ? 0 : 1;
        double half = 0.5 * (p.delta - d);
        for (size_t i = 0; i < gx.size(); i++) {
            double s = d + half * (gx[i] + 1.0);
            double wi = half * gw[i] * (1.0 - win->phi(s));
            double y = s / p.dt;
            int lo = (int)std::floor(y) - p.p / 2 + 1;
            lo = std::max(lo, m_min);
            lo = std::min(lo, p.m_max - p.p + 1);
            // barycentric weights at y for nodes lo .. lo+p-1
            int hit = -1;
            double den = 0.0, tmp[32];
            for (int r = 0; r < p.p; r++) {
                double dy = y - (double)(lo + r);
                if (dy == 0.0) { hit = r; break; }
                tmp[r] = lam[r] / dy;
                den += tmp[r];
            }
            if (hit >= 0) {
                Q[lo + hit] += wi;
            } else {
                for (int r = 0; r < p.p; r++) Q[lo + r] += wi * tmp[r] / den;
            }
        }
        return true;
    }
};

// all (target, source) pairs with distance < delta, sources sorted; periodic images folded
void find_pairs(const std::vector<double>& xt, const std::vector<double>& xs, double radius,
                bool periodic, std::vector<std::vector<std::pair<int32_t, double>>>& out) {
    int64_t T = (int64_t)xt.size();
    int64_t S = (int64_t)xs.size();
    out.assign(T, {});
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            auto& lst = out[j];
            for (int img = -1; img <= 1; img++) {
                if (!periodic && img != 0) continue;
                double shift = 2.0 * kPi * img;
                double lo = xt[j] - radius - shift, hi = xt[j] + radius - shift;
                auto it = std::lower_bound(xs.begin(), xs.end(), lo);
                for (; it != xs.end() && *it <= hi; ++it) {
                    int64_t l = it - xs.begin();
                    double d = std::fabs(xt[j] - (xs[l] + shift));
                    if (d < radius) lst.emplace_back((int32_t)l, d);
                }
            }
            std::sort(lst.begin(), lst.end(),
                      [](const std::pair<int32_t, double>& u, const std::pair<int32_t, double>& v) {
                          return u.first < v.first || (u.first == v.first && u.second < v.second);
                      });
            (void)S;
        }
    });
}

int build_local(const Params& P, const Window& win, const std::vector<double>& xt,
                const std::vector<double>& xs, bool include_m0, LocalCSR& csr,
                std::vector<std::vector<std::pair<int32_t, double>>>* nearby_out,
                int64_t max_bytes, std::string& err) {
    LocalRule rule;
    rule.init(P, win);
    std::vector<std::vector<std::pair<int32_t, double>>> pairs;
    find_pairs(xt, xs, P.delta, P.bc == WAVE1D_PERIODIC, pairs);
    int64_t T = (int64_t)xt.size();
    csr.row_ptr.assign(T + 1, 0);
    for (int64_t j = 0; j < T; j++) csr.row_ptr[j + 1] = csr.row_ptr[j] + (int64_t)pairs[j].size();
    int64_t np = csr.row_ptr[T];
    csr.src.assign(np, 0);
    csr.mrange.assign(np, 0);
    csr.woff.assign(np + 1, 0);
    // first pass: each pair's weights and their non-zero m range.  Where even m_max + 1 weights per
    // pair fit the budget the weights are kept per row and copied into place afterwards; otherwise
    // (the budget may refuse the layout) only the ranges are kept and a second pass recomputes them.
    const bool keep = (double)np * (double)(P.m_max + 1) * 8.0 <= (double)max_bytes;
    std::vector<std::vector<double>> rowbuf(keep ? T : 0);
    std::vector<int32_t> lo(np), cnt(np);
    std::atomic<int64_t> nearby{0};
    parallel_for(T, [&](int64_t a, int64_t b) {
        std::vector<double> Q(P.m_max + 1);
        int64_t nb = 0;
        for (int64_t j = a; j < b; j++) {
            for (size_t e = 0; e < pairs[j].size(); e++) {
                int64_t q = csr.row_ptr[j] + (int64_t)e;
                double d = pairs[j][e].second;
                csr.src[q] = pairs[j][e].first;
                rule.weights(d, Q.data());
                int m0 = include_m0 ? 0 : 1;
                int first = -1, last = -1;
                for (int m = m0; m <= P.m_max; m++)
                    if (Q[m] != 0.0) { if (first < 0) first = m; last = m; }
                if (first < 0) { first = m0; last = m0 - 1; }
                lo[q] = first;
                cnt[q] = last - first + 1;
                if (keep) rowbuf[j].insert(rowbuf[j].end(), Q.begin() + first, Q.begin() + last + 1);
                if (d < P.dt) nb++;
            }
        }
        nearby += nb;
    });
    csr.nearby = nearby.load();
    for (int64_t q = 0; q < np; q++) {
        csr.woff[q + 1] = csr.woff[q] + cnt[q];
        csr.mrange[q] = lo[q] | (cnt[q] << 16);
    }
    int64_t nw = csr.woff[np];
    if ((double)nw * 8.0 > (double)max_bytes) {
        err = "local weights need " + std::to_string(nw * 8) + " bytes, over the budget max_local_bytes";
        return WAVE1D_ENOMEM;
    }
    csr.w.assign(nw, 0.0);
    parallel_for(T, [&](int64_t a, int64_t b) {
        std::vector<double> Q(P.m_max + 1);
        for (int64_t j = a; j < b; j++) {
            if (keep) {
                if (!rowbuf[j].empty())
                    std::copy(rowbuf[j].begin(), rowbuf[j].end(), csr.w.begin() + csr.woff[csr.row_ptr[j]]);
                std::vector<double>().swap(rowbuf[j]);
                continue;
            }
            for (size_t e = 0; e < pairs[j].size(); e++) {
                int64_t q = csr.row_ptr[j] + (int64_t)e;
                rule.weights(pairs[j][e].second, Q.data());
                for (int c = 0; c < cnt[q]; c++) csr.w[csr.woff[q] + c] = Q[lo[q] + c];
            }
        }
    });
    if (nearby_out) {
        nearby_out->assign(T, {});
        for (int64_t j = 0; j < T; j++)
            for (auto& pr : pairs[j])
                if (pr.second < P.dt) (*nearby_out)[j].push_back(pr);
    }
    return WAVE1D_OK;
}

// Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix (in place into inv)
bool invert(int n, std::vector<double>& A, double* inv) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int j = 0; j < n; j++) {
                std::swap(A[c * n + j], A[piv * n + j]);
                std::swap(inv[c * n + j], inv[piv * n + j]);
            }
        }
        double d = 1.0 / A[c * n + c];
        for (int j = 0; j < n; j++) { A[c * n + j] *= d; inv[c * n + j] *= d; }
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; j++) { A[r * n + j] -= f * A[c * n + j]; inv[r * n + j] -= f * inv[c * n + j]; }
        }
    }
    return true;
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// Kaiser-Bessel spreading weights of points x (the kernel of eq. KB on the fine grid): first grid
// index (wrapped) and w weights per point
void spread_weights(const Params& P, const std::vector<double>& x, std::vector<int32_t>& i0,
                    std::vector<double>& ker) {
    int64_t n = (int64_t)x.size();
    int w = P.nufft_w;
    i0.assign(n, 0);
    ker.assign(n * w, 0.0);
    double inv_i0b = 1.0 / bessel_i0(P.kb_beta);
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            double u = (x[j] + kPi) / P.h_f;
            int64_t first = (int64_t)std::ceil(u - 0.5 * w);
            for (int t = 0; t < w; t++) {
                double z = (double)(first + t - u) * 2.0 / w;
                double r = 1.0 - z * z;
                ker[j * w + t] = r > 0.0 ? bessel_i0(P.kb_beta * std::sqrt(r)) * inv_i0b : 0.0;
            }
            int64_t c = first % P.nf;
            if (c < 0) c += P.nf;
            i0[j] = (int32_t)c;
        }
    });
}

// NUFFT deconvolution folded with the real-FFT pre/post-processing, per mode k = 0..K:
//   psihat(k) = w h sinh(r)/r / I0(beta), r = sqrt(beta^2 - (k w h/2)^2)  (transform of eq. KB)
//   modefac[k][0..2]: type-1 (deconv1 and deconv1 e^{2 pi i k/nf}); [3..6]: type-2 spectrum
void nufft_factors(const Params& P, std::vector<double>& deconv1, std::vector<double>& deconv2,
                   std::vector<double>& modefac) {
    const int K1 = P.K + 1;
    deconv1.assign(K1, 0.0);
    deconv2.assign(K1, 0.0);
    double i0b = bessel_i0(P.kb_beta);
    for (int k = 0; k < K1; k++) {
        double om = 0.5 * k * P.nufft_w * P.h_f;
        double r = std::sqrt(P.kb_beta * P.kb_beta - om * om);
        double ph = P.nufft_w * P.h_f * (r > 0 ? std::sinh(r) / r : 1.0) / i0b;
        double sgn = (k % 2 == 0) ? 1.0 : -1.0;
        deconv1[k] = sgn * P.h_f / (2.0 * kPi * ph);
        deconv2[k] = sgn * P.h_f / ph;
    }
    modefac.assign((size_t)K1 * 8, 0.0);
    for (int k = 0; k < K1; k++) {
        double a1 = 2.0 * kPi * (double)k / (double)P.nf;          // e^{+i a1} = w^k
        double a2 = 2.0 * kPi * (double)(P.L - k) / (double)P.nf;  // e^{-i a2} = w'^{L-k}
        double d1 = deconv1[k], d2 = deconv2[k];
        double* f = &modefac[(size_t)k * 8];
        f[0] = d1;
        f[1] = d1 * std::cos(a1);
        f[2] = d1 * std::sin(a1);
        // 1 + i e^{-i a1} = (1 + sin a1) + i cos a1
        f[3] = d2 * (1.0 + std::sin(a1));
        f[4] = d2 * std::cos(a1);
        // 1 - i e^{-i a2} = (1 - sin a2) - i cos a2
        f[5] = d2 * (1.0 - std::sin(a2));
        f[6] = -d2 * std::cos(a2);
    }
}

// fine grid and kernel for N_F = 2K + 1 modes at tolerance tol (w taps unless w_in > 0)
void nufft_grid(Params& P, int K, double tol, int w_in) {
    P.K = K;
    P.nf = 1;
    while (P.nf < 2 * (2 * K + 1)) P.nf <<= 1;
    if (P.nf < 64) P.nf = 64;
    P.L = P.nf / 2;
    int lg = 0;
    while ((1 << lg) < P.L) lg++;
    P.L1 = 1 << ((lg + 1) / 2);          // L1 >= L2: balances column and row-pair passes
    P.L2 = P.L / P.L1;
    P.h_f = 2.0 * kPi / P.nf;
    P.nufft_w = w_in > 0 ? w_in : (int)std::ceil(std::log10(1.0 / tol)) + 1;
    P.nufft_w = std::max(4, std::min(16, P.nufft_w));
    double upsamp = (double)P.nf / (2.0 * P.K + 1.0);
    P.kb_beta = kPi * P.nufft_w * (1.0 - 1.0 / (2.0 * upsamp));
}

void nufft_ranges(const std::vector<int32_t>& i0, const int64_t* offsets, int n_inst, int nf, int w,
                  int max_cells, int max_points, int empty_cells, int threads, std::vector<NuRange>& ranges,
                  std::vector<int32_t>& runs) {
    ranges.clear();
    runs.clear();
    std::vector<int32_t> ps(nf + 1);
    for (int b = 0; b < n_inst; b++) {
        const int64_t o = offsets[b], mb = offsets[b + 1] - o;
        std::fill(ps.begin(), ps.end(), 0);
        for (int64_t i = 0; i < mb; i++) ps[i0[o + i] + 1]++;
        for (int f = 0; f < nf; f++) ps[f + 1] += ps[f];
        auto pts = [&](int f0, int f1) {              // points whose first cell is in [f0, f1), f0 may be < 0
            if (f0 >= 0) return ps[f1] - ps[f0];
            return (ps[nf] - ps[nf + f0]) + ps[f1];
        };
        for (int c0 = 0; c0 < nf;) {
            int c1 = c0 + 1;
            if (pts(c0 - w + 1, c0 + 1) == 0) {
                while (c1 < nf && c1 - c0 < empty_cells && pts(c1 - w + 1, c1 + 1) == 0) c1++;
            } else {
                while (c1 < nf && c1 - c0 < max_cells && pts(c0 - w + 1, c1 + 1) <= max_points) c1++;
            }
            NuRange r{};
            r.c0 = b * nf + c0;
            r.nc = c1 - c0;
            const int h0 = c0 - w + 1;                // first halo cell (negative: wraps to the end)
            if (h0 >= 0) {
                r.a0 = (int32_t)(o + ps[h0]);
                r.na = ps[c1] - ps[h0];
                r.b0 = (int32_t)o;
                r.nb = 0;
            } else {
                r.a0 = (int32_t)(o + ps[nf + h0]);
                r.na = ps[nf] - ps[nf + h0];
                r.b0 = (int32_t)o;
                r.nb = ps[c1];
            }
            r.roff = (int32_t)runs.size();
            if (r.na + r.nb > 0) {
                for (int k = 0; k <= r.nc + w - 1; k++) {    // run starts in staging order, then the end
                    const int f = h0 + k;
                    int off;
                    if (k == r.nc + w - 1) off = r.na + r.nb;
                    else if (f >= 0) off = (h0 >= 0 ? ps[f] - ps[h0] : r.na + ps[f]);
                    else off = ps[nf + f] - ps[nf + h0];
                    runs.push_back(off);
                }
            }
            const int nr = r.nc + w - 1;
            r.lg = 0;
            while (r.lg < 5 && (nr << (r.lg + 1)) <= threads) r.lg++;
            ranges.push_back(r);
            c0 = c1;
        }
    }
}

namespace {
int build_local_and_blocks(const Params& P, const Window& win, HostPlan& hp, int max_block,
                           int64_t max_local_bytes, std::string& err);
void range_windows(HostPlan& hp);
}  // namespace

// W = 2 b / (pi gamma) rounded up, b = ln(1/tol) (eqs. b, W), unless given
int window_steps(double tol, double gamma, int W) {
    return W > 0 ? W : (int)std::ceil(2.0 * std::log(1.0 / tol) / (kPi * gamma));
}

// The range tables depend on dt, delta, b, W, N_L, m_max and p only (and the interval cap), so plans
// that share them (the instances of a batched plan) build them once: the last few are kept.
static void range_tables_cached(const Params& P, RangeTables& rt) {
    struct Entry {
        double dt, delta, b, cap;
        int W, NL, m_max, p;
        RangeTables rt;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    const char* env = std::getenv("WAVE1D_RANGE_WIDTH");
    const double cap = env ? std::atof(env) : -1.0;
    auto same = [&](const Entry& e) {
        return e.dt == P.dt && e.delta == P.delta && e.b == P.b && e.cap == cap && e.W == P.W && e.NL == P.NL &&
               e.m_max == P.m_max && e.p == P.p;
    };
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry& e : cache)
            if (same(e)) {
                rt = e.rt;
                return;
            }
    }
    build_range_tables(P, rt);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 4) cache.erase(cache.begin());
    cache.push_back(Entry{P.dt, P.delta, P.b, cap, P.W, P.NL, P.m_max, P.p, rt});
}

// History tables (eqs. pkqkcomp, hkcompdisc, the mode rotation, the NUFFT deconvolution, the FFT
// twiddles): functions of dt, K, W, N_g, the window and the fine grid alone, so plans that share
// them (the instances of a batched plan) compute them once; the last few are kept.
static void history_tables_build(const Params& P, const Window& win, HostPlan& hp) {
    const double dt = P.dt;
    std::vector<double> gx, gw;
    gauss_legendre(P.Ng, gx, gw);
    int K1 = P.K + 1;
    std::vector<double> mu(P.Ng), wt(P.Ng), d1(P.W * P.Ng), d2(P.W * P.Ng);
    for (int g = 0; g < P.Ng; g++) {
        mu[g] = 0.5 * dt * (gx[g] + 1.0);
        wt[g] = 0.5 * dt * gw[g];
    }
    for (int m = 0; m < P.W; m++)
        for (int g = 0; g < P.Ng; g++) {
            double tau = m * dt + mu[g];
            d1[m * P.Ng + g] = win.dphi(tau);
            d2[m * P.Ng + g] = win.ddphi(tau);
        }
    hp.pq.assign((size_t)P.W * K1 * 2, 0.0);
    parallel_for(K1, [&](int64_t a, int64_t b) {
        for (int64_t k = a; k < b; k++) {
            double kd = (double)k;
            for (int m = 0; m < P.W; m++) {
                double sp = 0.0, sq = 0.0;
                for (int g = 0; g < P.Ng; g++) {
                    double tau = m * dt + mu[g];
                    double psi = 2.0 * std::cos(kd * tau) * d1[m * P.Ng + g] +
                                 sinc_k(kd, tau) * d2[m * P.Ng + g];       // eq. psidef
                    sp += wt[g] * sinc_k(kd, dt - mu[g]) * psi;
                    sq += wt[g] * std::cos(kd * (dt - mu[g])) * psi;
                }
                hp.pq[((size_t)m * K1 + k) * 2 + 0] = dt * sp;               // eq. hkcompdisc
                hp.pq[((size_t)m * K1 + k) * 2 + 1] = dt * sq;
            }
        }
    });
    hp.rot.assign((size_t)K1 * 3, 0.0);
    for (int k = 0; k < K1; k++) {
        hp.rot[k * 3 + 0] = std::cos(k * dt);
        hp.rot[k * 3 + 1] = sinc_k(k, dt);
        hp.rot[k * 3 + 2] = k * std::sin(k * dt);
    }
    std::vector<double> modefac;
    nufft_factors(P, hp.deconv1, hp.deconv2, modefac);
    hp.twiddle.assign((size_t)P.L * 2, 0.0);
    for (int j = 0; j < P.L; j++) {
        double a = 2.0 * kPi * (double)j / (double)P.L;
        hp.twiddle[2 * j] = std::cos(a);
        hp.twiddle[2 * j + 1] = std::sin(a);
    }
    // per-mode factors of the real-FFT post/pre-processing folded with the deconvolution
    hp.modefac = modefac;
    hp.tw2K.assign((size_t)4 * P.K, 0.0);
    for (int a = 0; a < 2 * P.K; a++) {
        double ang = kPi * (double)a / (double)P.K;
        hp.tw2K[2 * a] = std::cos(ang);
        hp.tw2K[2 * a + 1] = std::sin(ang);
    }
}

static void history_tables(const Params& P, const Window& win, HostPlan& hp) {
    struct Entry {
        double dt, b, delta, kb_beta;
        int K, W, Ng, nf, L, nufft_w;
        std::vector<double> pq, rot, deconv1, deconv2, twiddle, modefac, tw2K;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    auto same = [&](const Entry& e) {
        return e.dt == P.dt && e.b == P.b && e.delta == P.delta && e.kb_beta == P.kb_beta && e.K == P.K &&
               e.W == P.W && e.Ng == P.Ng && e.nf == P.nf && e.L == P.L && e.nufft_w == P.nufft_w;
    };
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry& e : cache)
            if (same(e)) {
                hp.pq = e.pq;
                hp.rot = e.rot;
                hp.deconv1 = e.deconv1;
                hp.deconv2 = e.deconv2;
                hp.twiddle = e.twiddle;
                hp.modefac = e.modefac;
                hp.tw2K = e.tw2K;
                return;
            }
    }
    history_tables_build(P, win, hp);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 4) cache.erase(cache.begin());
    cache.push_back(Entry{P.dt, P.b, P.delta, P.kb_beta, P.K, P.W, P.Ng, P.nf, P.L, P.nufft_w, hp.pq, hp.rot,
                          hp.deconv1, hp.deconv2, hp.twiddle, hp.modefac, hp.tw2K});
}

// ---------------------------------------------------------------------------------------------
int build_host_plan(const double* x_in, const double* beta_in, int64_t M, int bc, double dt,
                    int64_t Nt, double tol, int p, double gamma, int W, int NL, int Ng, int nufft_w,
                    int rbc_period, int max_block, int64_t max_local_bytes, HostPlan& hp,
                    std::string& err, bool range) {
    Params& P = hp.P;
    P.M = M;
    P.Nt = Nt;
    P.bc = bc;
    P.dt = dt;
    P.tol = tol;
    P.p = p;
    P.gamma = gamma;
    P.b = std::log(1.0 / tol);                                        // eq. b
    P.K = (int)std::floor(kPi / dt);                                  // eq. Kdt (floor)
    P.W = window_steps(tol, gamma, W);
    P.delta = P.W * dt;                                               // eq. W
    P.m_max = P.W + (p + 1) / 2;                                      // Sec. 4.1
    P.NL = NL > 0 ? NL : P.W;                                         // Sec. 4.3
    P.Ng = Ng > 0 ? Ng : 32;
    P.ring = P.m_max + 1;
    if (P.K < 2) { err = "dt too large: K = floor(pi/dt) < 2"; return WAVE1D_EINVAL; }
    if (!(P.delta < kPi)) { err = "window delta = W dt must be below pi (Sec. 3)"; return WAVE1D_EDOMAIN; }
    if (P.m_max - p + 1 < 1) { err = "window too short for the interpolation order"; return WAVE1D_EINVAL; }
    // radiation projection grid (Sec. 4.4)
    P.h_rbc = kPi / P.K;
    P.delta_s = P.W * P.h_rbc;
    P.rbc_period = rbc_period > 0 ? rbc_period : (int)std::ceil(1.5 * P.W);
    if (bc == WAVE1D_FREE && 4 * P.W >= 2 * P.K) { err = "K too small for the radiation projection (4W >= 2K)"; return WAVE1D_EDOMAIN; }
    // NUFFT fine grid: power of two, at least twice N_F
    P.nf = (int)next_pow2(2 * (2 * (int64_t)P.K + 1));
    if (P.nf < 64) P.nf = 64;
    P.L = P.nf / 2;
    int lg = 0;
    while ((1 << lg) < P.L) lg++;
    P.L1 = 1 << ((lg + 1) / 2);          // L1 >= L2: balances column and row-pair passes
    P.L2 = P.L / P.L1;
    if (P.L2 > 1024) { err = "fine grid too large for this build (nf > 2^21)"; return WAVE1D_EUNSUPPORTED; }
    P.h_f = 2.0 * kPi / P.nf;
    P.nufft_w = nufft_w > 0 ? nufft_w : (int)std::ceil(std::log10(1.0 / tol)) + 1;
    P.nufft_w = std::max(4, std::min(16, P.nufft_w));
    double upsamp = (double)P.nf / (2.0 * P.K + 1.0);
    P.kb_beta = kPi * P.nufft_w * (1.0 - 1.0 / (2.0 * upsamp));

    // positions: wrap (periodic) or check Omega (free space), then sort
    std::vector<double> xw(M);
    double omega_lim = kPi - 3.0 * std::max(P.delta, P.delta_s);
    for (int64_t j = 0; j < M; j++) {
        double v = x_in[j];
        if (!std::isfinite(v) || !std::isfinite(beta_in[j]) || beta_in[j] < 0.0) {
            err = "non-finite position or negative/non-finite stiffness";
            return WAVE1D_EINVAL;
        }
        if (bc == WAVE1D_PERIODIC) {
            v = std::fmod(v + kPi, 2.0 * kPi);
            if (v < 0) v += 2.0 * kPi;
            v -= kPi;
            if (v >= kPi) v -= 2.0 * kPi;
        } else if (std::fabs(v) > omega_lim) {
            err = "free-space spring outside Omega = [-pi + 3 delta, pi - 3 delta] (Sec. 4.4)";
            return WAVE1D_EDOMAIN;
        }
        xw[j] = v;
    }
    hp.perm.resize(M);
    std::iota(hp.perm.begin(), hp.perm.end(), 0);
    std::stable_sort(hp.perm.begin(), hp.perm.end(), [&](int32_t a, int32_t b) { return xw[a] < xw[b]; });
    hp.x.resize(M);
    hp.beta.resize(M);
    for (int64_t j = 0; j < M; j++) {
        hp.x[j] = xw[hp.perm[j]];
        hp.beta[j] = beta_in[hp.perm[j]];
    }

    Window win(P.delta, P.b);

    // history kernels p_k, q_k (eq. pkqkcomp) with Ng-point Gauss-Legendre, dt folded in
    history_tables(P, win, hp);

    // spreading weights and bins by first grid index
    spread_weights(P, hp.x, hp.sp_i0, hp.sp_ker);
    hp.bin_ptr.assign(P.nf + 1, 0);
    for (int64_t j = 0; j < M; j++) hp.bin_ptr[hp.sp_i0[j] + 1]++;
    for (int c = 0; c < P.nf; c++) hp.bin_ptr[c + 1] += hp.bin_ptr[c];
    hp.bin_list.assign(M, 0);
    {
        std::vector<int32_t> fill(hp.bin_ptr.begin(), hp.bin_ptr.end() - 1);
        for (int64_t j = 0; j < M; j++) hp.bin_list[fill[hp.sp_i0[j]]++] = (int32_t)j;
    }
    // spreading as a sparse matrix, G[i] = sum_e g_w[e] sigma_{g_src[e]}, its rows in the order the
    // column pass of the FFT reads them: real i = 2 r + h of complex point r = i2 + L2 i1 is row
    // c = 2 (i2 L1 + i1) + h, so each column's entries form one contiguous range
    {
        int w = P.nufft_w;
        auto row_of = [&](int i) {
            int r = i >> 1, h = i & 1;
            return 2 * ((r % P.L2) * P.L1 + r / P.L2) + h;
        };
        hp.g_ptr.assign(P.nf + 1, 0);
        for (int64_t j = 0; j < M; j++)
            for (int t = 0; t < w; t++) hp.g_ptr[row_of((hp.sp_i0[j] + t) % P.nf) + 1]++;
        for (int i = 0; i < P.nf; i++) hp.g_ptr[i + 1] += hp.g_ptr[i];
        hp.g_src.assign((size_t)M * w, 0);
        hp.g_w.assign((size_t)M * w, 0.0);
        std::vector<int32_t> fill(hp.g_ptr.begin(), hp.g_ptr.end() - 1);
        for (int64_t j = 0; j < M; j++)
            for (int t = 0; t < w; t++) {
                int c = row_of((hp.sp_i0[j] + t) % P.nf);
                hp.g_src[fill[c]] = (int32_t)j;
                hp.g_w[fill[c]] = hp.sp_ker[j * w + t];
                fill[c]++;
            }
    }

    if (range) {
        // no pair lists: index windows, the weights as polynomials of the distance
        hp.range = true;
        range_tables_cached(P, hp.rt);
        range_windows(hp);
    } else {
        int rc = build_local_and_blocks(P, win, hp, max_block, max_local_bytes, err);
        if (rc) return rc;
    }

    // radiation projection tables (Sec. 4.4): grid x_i = i h (i < K), (i - 2K) h (i >= K)
    if (bc == WAVE1D_FREE) {
        Window swin(P.delta_s, P.b);
        hp.rbc_idx.clear();
        hp.rbc_x.clear();
        hp.rbc_phi.clear();
        hp.rbc_dphi.clear();
        for (int i = P.K - 2 * P.W; i < P.K; i++) {
            double xg = i * P.h_rbc, arg = kPi - P.delta_s - xg;
            hp.rbc_idx.push_back(i);
            hp.rbc_x.push_back(xg);
            hp.rbc_phi.push_back(swin.phi(arg));
            hp.rbc_dphi.push_back(swin.dphi(arg));
        }
        for (int i = P.K; i < P.K + 2 * P.W; i++) {
            double xg = (i - 2 * P.K) * P.h_rbc, arg = kPi - P.delta_s + xg;
            hp.rbc_idx.push_back(i);
            hp.rbc_x.push_back(xg);
            hp.rbc_phi.push_back(swin.phi(arg));
            hp.rbc_dphi.push_back(swin.dphi(arg));
        }
    }
    return WAVE1D_OK;
}

namespace {
// Local part (Sec. 4.1) with stored weights and the inverted blocks of springs closer than dt
// (eq. linearSystem).
int build_local_and_blocks(const Params& P, const Window& win, HostPlan& hp, int max_block,
                           int64_t max_local_bytes, std::string& err) {
    const int64_t M = P.M;
    std::vector<std::vector<std::pair<int32_t, double>>> nearby;
    int rc = build_local(P, win, hp.x, hp.x, false, hp.loc, &nearby, max_local_bytes, err);
    if (rc) return rc;
    if ((rc = build_rows(hp.loc, 1, hp.lrows, err))) return rc;
    build_items(hp.lrows, hp.litems);
    {
        std::vector<int32_t> parent(M);
        std::iota(parent.begin(), parent.end(), 0);
        std::function<int32_t(int32_t)> find = [&](int32_t i) {
            while (parent[i] != i) { parent[i] = parent[parent[i]]; i = parent[i]; }
            return i;
        };
        for (int64_t j = 0; j < M; j++)
            for (auto& pr : nearby[j]) {
                int32_t a = find((int32_t)j), b = find(pr.first);
                if (a != b) parent[a] = b;
            }
        std::vector<int64_t> cnt(M + 1, 0);
        for (int64_t j = 0; j < M; j++) cnt[find((int32_t)j) + 1]++;
        std::vector<int32_t> roots;
        for (int64_t r = 0; r < M; r++) if (cnt[r + 1] > 0) roots.push_back((int32_t)r);
        std::vector<int64_t> rid(M, -1);
        for (size_t i = 0; i < roots.size(); i++) rid[roots[i]] = (int64_t)i;
        int64_t nb = (int64_t)roots.size();
        hp.blk_ptr.assign(nb + 1, 0);
        for (int64_t j = 0; j < M; j++) hp.blk_ptr[rid[find((int32_t)j)] + 1]++;
        for (int64_t b = 0; b < nb; b++) hp.blk_ptr[b + 1] += hp.blk_ptr[b];
        hp.blk_members.assign(M, 0);
        std::vector<int64_t> fill(hp.blk_ptr.begin(), hp.blk_ptr.end() - 1);
        std::vector<int32_t> local_of(M);
        for (int64_t j = 0; j < M; j++) {
            int64_t b = rid[find((int32_t)j)];
            local_of[j] = (int32_t)(fill[b] - hp.blk_ptr[b]);
            hp.blk_members[fill[b]++] = (int32_t)j;
        }
        hp.blk_inv_off.assign(nb + 1, 0);
        hp.max_block = 0;
        for (int64_t b = 0; b < nb; b++) {
            int64_t s = hp.blk_ptr[b + 1] - hp.blk_ptr[b];
            hp.max_block = std::max(hp.max_block, s);
            hp.blk_inv_off[b + 1] = hp.blk_inv_off[b] + s * s;
        }
        if (hp.max_block > max_block) {
            err = "a block of springs closer than dt has " + std::to_string(hp.max_block) +
                  " members, above max_block; the direct block solve of this build does not cover it";
            return WAVE1D_EUNSUPPORTED;
        }
        hp.inv.assign(hp.blk_inv_off[nb], 0.0);
        LocalRule rule;
        rule.init(P, win);
        std::atomic<int> bad{0};
        parallel_for(nb, [&](int64_t a, int64_t bb) {
            std::vector<double> A, Q(P.m_max + 1);
            for (int64_t b = a; b < bb; b++) {
                int64_t s = hp.blk_ptr[b + 1] - hp.blk_ptr[b];
                A.assign(s * s, 0.0);
                for (int64_t i = 0; i < s; i++) {
                    int32_t j = hp.blk_members[hp.blk_ptr[b] + i];
                    A[i * s + i] += 1.0;
                    for (auto& pr : nearby[j]) {
                        rule.weights(pr.second, Q.data());
                        A[i * s + local_of[pr.first]] += 0.5 * hp.beta[j] * Q[0];
                    }
                }
                std::vector<double> inv_rm(s * s);
                if (!invert((int)s, A, inv_rm.data())) bad = 1;
                // stored column-major: inv[l * s + i] = (I + S)^{-1}[i][l]
                double* dst = &hp.inv[hp.blk_inv_off[b]];
                for (int64_t i = 0; i < s; i++)
                    for (int64_t l = 0; l < s; l++) dst[l * s + i] = inv_rm[i * s + l];
            }
        });
        if (bad) { err = "singular block of I + S"; return WAVE1D_EINVAL; }
        // pack consecutive blocks of at most 32 members into warps of 32 lanes; larger blocks
        // are split into tasks of 32 rows (one task above 256 members)
        hp.sg_j.clear();
        hp.sg_meta.clear();
        hp.sg_off.clear();
        hp.sg_beta.clear();
        hp.sg_ip.clear();
        hp.sg_icnt.clear();
        hp.sg_smax.clear();
        hp.big_blk.clear();
        hp.big_row0.clear();
        int used = 32;
        for (int64_t b = 0; b < nb; b++) {
            int64_t sz = hp.blk_ptr[b + 1] - hp.blk_ptr[b];
            if (sz > 32) {
                for (int64_t r0 = 0; r0 < sz; r0 += 32) {
                    hp.big_blk.push_back(b);
                    hp.big_row0.push_back((int32_t)r0);
                    if (sz > 256) break;
                }
                continue;
            }
            if (used + sz > 32) {
                hp.sg_j.insert(hp.sg_j.end(), 32, -1);
                hp.sg_meta.insert(hp.sg_meta.end(), 32, 0);
                hp.sg_off.insert(hp.sg_off.end(), 32, 0);
                hp.sg_beta.insert(hp.sg_beta.end(), 32, 0.0);
                hp.sg_ip.insert(hp.sg_ip.end(), 32, 0);
                hp.sg_icnt.insert(hp.sg_icnt.end(), 32, 0);
                hp.sg_smax.push_back(0);
                used = 0;
            }
            size_t g = hp.sg_smax.size() - 1;
            for (int64_t i = 0; i < sz; i++) {
                size_t lane = g * 32 + used + i;
                int32_t j = hp.blk_members[hp.blk_ptr[b] + i];
                hp.sg_j[lane] = j;
                hp.sg_meta[lane] = used | (int)(sz << 8) | (int)(i << 16);
                hp.sg_off[lane] = hp.blk_inv_off[b];
                hp.sg_beta[lane] = hp.beta[j];
                hp.sg_ip[lane] = hp.litems.item_ptr[j];
                hp.sg_icnt[lane] = (int32_t)(hp.litems.item_ptr[j + 1] - hp.litems.item_ptr[j]);
            }
            hp.sg_smax[g] = std::max<int32_t>(hp.sg_smax[g], (int32_t)sz);
            used += (int)sz;
        }
    }
    return WAVE1D_OK;
}

// position of extended source index e (periodic: spring e mod M shifted by 2 pi floor(e / M));
// every window test of the range mode uses this expression, on the host and on the device
inline double x_ext(const std::vector<double>& x, int64_t M, int64_t e) {
    if (e < 0) return x[e + M] - 2.0 * kPi;
    if (e >= M) return x[e - M] + 2.0 * kPi;
    return x[e];
}

// first extended index in [lo, hi) whose position satisfies pred (pred false .. true in index order)
template <class F>
int64_t first_true(int64_t lo, int64_t hi, F pred) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (pred(mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Index windows of the range mode: per spring the sources closer than dt (the implicit block of
// eq. linearSystem, decided by |x_e - x_j| < dt in FP64 exactly as the device evaluates it), and
// per block of kRsTargets targets the sources within delta of any of them (a superset: the device
// decides each pair from the float-pair positions).
void range_windows(HostPlan& hp) {
    const Params& P = hp.P;
    const int64_t M = P.M;
    const bool per = P.bc == WAVE1D_PERIODIC;
    const int64_t elo = per ? -M : 0, ehi = per ? 2 * M : M;
    const std::vector<double>& x = hp.x;
    hp.nb_lo.assign(M, 0);
    hp.nb_cnt.assign(M, 0);
    parallel_for(M, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            // |x_e - x_j| < dt is monotone on each side of j
            const int64_t lo = first_true(std::max(elo, j - M), j + 1,
                                          [&](int64_t e) { return std::fabs(x_ext(x, M, e) - x[j]) < P.dt; });
            const int64_t hi = first_true(j, std::min(ehi, j + M),
                                          [&](int64_t e) { return !(std::fabs(x_ext(x, M, e) - x[j]) < P.dt); });
            hp.nb_lo[j] = (int32_t)lo;
            hp.nb_cnt[j] = (int32_t)(hi - lo);
        }
    });
    hp.nb_off.assign(M + 1, 0);
    for (int64_t j = 0; j < M; j++) hp.nb_off[j + 1] = hp.nb_off[j] + hp.nb_cnt[j];
    // pairs closer than delta (reported; the device never lists them)
    std::vector<int64_t> cnt(M, 0);
    parallel_for(M, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            const int64_t lo = first_true(std::max(elo, j - M), j + 1,
                                          [&](int64_t e) { return std::fabs(x_ext(x, M, e) - x[j]) < P.delta; });
            const int64_t hi = first_true(j, std::min(ehi, j + M),
                                          [&](int64_t e) { return !(std::fabs(x_ext(x, M, e) - x[j]) < P.delta); });
            cnt[j] = hi - lo;
        }
    });
    hp.range_pairs = 0;
    for (int64_t j = 0; j < M; j++) hp.range_pairs += cnt[j];
    const int64_t nblk = (M + kRsTargets - 1) / kRsTargets;
    const double reach = P.delta * (1.0 + 1e-12) + 1e-13;
    hp.blk_win.assign(4 * nblk, 0);
    for (int64_t b = 0; b < nblk; b++) {
        const int64_t j0 = b * kRsTargets, j1 = std::min(M, j0 + kRsTargets) - 1;
        const double xa = x[j0], xb = x[j1];
        hp.blk_win[4 * b + 0] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(x, M, e) > xa - reach; });
        hp.blk_win[4 * b + 1] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(x, M, e) >= xa; });
        hp.blk_win[4 * b + 2] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(x, M, e) > xb; });
        hp.blk_win[4 * b + 3] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(x, M, e) >= xb + reach; });
    }
}
}  // namespace

// Regroup CSR local weights into m-major rows (see LocalRows).  Within a row the sources are
// sorted by (m_lo, source); for each m the active sources are those with m_lo <= m, a prefix.
// Entries with m above a source's last weight are stored as zeros.
int build_rows(const LocalCSR& csr, int m_first, LocalRows& rows, std::string& err) {
    int64_t T = (int64_t)csr.row_ptr.size() - 1;
    int m_top = m_first;
    for (size_t q = 0; q < csr.mrange.size(); q++) {
        int lo = csr.mrange[q] & 0xffff, cnt = csr.mrange[q] >> 16;
        if (cnt > 0) m_top = std::max(m_top, lo + cnt - 1);
    }
    rows.m_first = m_first;
    rows.nm = m_top - m_first + 1;
    rows.src_off.assign(T + 1, 0);
    rows.w_off.assign(T + 1, 0);
    rows.cnt.assign((size_t)T * rows.nm, 0);
    rows.src.assign(csr.src.size(), 0);
    std::vector<int64_t> nw(T, 0);
    std::vector<std::vector<int64_t>> order(T);
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            int64_t p0 = csr.row_ptr[j], p1 = csr.row_ptr[j + 1];
            auto& ord = order[j];
            ord.resize(p1 - p0);
            for (int64_t q = p0; q < p1; q++) ord[q - p0] = q;
            // sources by the first m they need; a source without weights (a pair inside delta by
            // rounding only, every Q_m zero) goes last, so the sources active at each m stay a
            // prefix of the list, which the counts below assume
            auto first_m = [&](int64_t q) {
                return (csr.mrange[q] >> 16) > 0 ? (csr.mrange[q] & 0xffff) : 0x7fffffff;
            };
            std::sort(ord.begin(), ord.end(), [&](int64_t u, int64_t v) {
                int lu = first_m(u), lv = first_m(v);
                return lu < lv || (lu == lv && csr.src[u] < csr.src[v]);
            });
            int64_t total = 0;
            for (int i = 0; i < rows.nm; i++) {
                int m = m_first + i;
                int64_t c = 0;
                for (int64_t q : ord) {
                    int lo = csr.mrange[q] & 0xffff, cnt = csr.mrange[q] >> 16;
                    if (cnt > 0 && lo <= m) c++;
                }
                if (c > 65535) c = -1;
                rows.cnt[(size_t)j * rows.nm + i] = (uint16_t)(c < 0 ? 0 : c);
                total += c;
            }
            nw[j] = total;
        }
    });
    for (int64_t j = 0; j < T; j++) {
        rows.src_off[j + 1] = rows.src_off[j] + (csr.row_ptr[j + 1] - csr.row_ptr[j]);
        rows.w_off[j + 1] = rows.w_off[j] + nw[j];
        if (csr.row_ptr[j + 1] - csr.row_ptr[j] > 65535) {
            err = "more than 65535 local neighbours of one target";
            return WAVE1D_EUNSUPPORTED;
        }
    }
    rows.w.assign(2 * (size_t)rows.w_off[T], 0.0f);
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            const auto& ord = order[j];
            for (size_t r = 0; r < ord.size(); r++) rows.src[rows.src_off[j] + r] = csr.src[ord[r]];
            int64_t off = rows.w_off[j];
            for (int i = 0; i < rows.nm; i++) {
                int m = m_first + i;
                int c = rows.cnt[(size_t)j * rows.nm + i];
                for (int r = 0; r < c; r++) {
                    int64_t q = ord[r];
                    int lo = csr.mrange[q] & 0xffff, cnt = csr.mrange[q] >> 16;
                    double v = (m >= lo && m < lo + cnt) ? csr.w[csr.woff[q] + (m - lo)] : 0.0;
                    float hi = (float)v;
                    float lo_part = (float)(v - (double)hi);
                    rows.w[2 * (off + r)] = hi;
                    rows.w[2 * (off + r) + 1] = lo_part;
                }
                off += c;
            }
        }
    });
    return WAVE1D_OK;
}

// Cut m-major rows into chunk items (see LocalItems).  Rank r of a row is active in slice i iff
// cnt[i] > r; cnt is non-decreasing in i, so rank r is active from first(r) on.  Elements are
// stored in pairs: elements 2u and 2u+1 of lane l sit at w[wbase + 64 u + 2 l + {0, 1}] (one
// 16-byte load per lane fetches both); len is rounded up to even with zero weights.
int build_items(const LocalRows& rows, LocalItems& it) {
    int64_t T = (int64_t)rows.src_off.size() - 1;
    int nm = rows.nm;
    it.m_first = rows.m_first;
    it.item_ptr.assign(T + 1, 0);
    for (int64_t j = 0; j < T; j++) {
        int64_t ns = rows.src_off[j + 1] - rows.src_off[j];
        it.item_ptr[j + 1] = it.item_ptr[j] + (ns + 31) / 32;
    }
    int64_t NI = it.item_ptr[T];
    it.row.assign(NI, 0);
    it.s0.assign(NI, 0);
    it.len.assign(NI, 0);
    it.wbase.assign(NI + 1, 0);
    it.src.assign(NI * 32, 0);
    for (int64_t j = 0; j < T; j++) {
        const uint16_t* cnt = &rows.cnt[(size_t)j * nm];
        for (int64_t c = it.item_ptr[j]; c < it.item_ptr[j + 1]; c++) {
            int r0 = (int)(32 * (c - it.item_ptr[j]));
            int first = nm;
            for (int i = 0; i < nm; i++)
                if (cnt[i] > r0) { first = i; break; }
            int len = nm - first;
            len += len & 1;
            it.row[c] = (int32_t)j;
            it.s0[c] = first;
            it.len[c] = len;
            it.wbase[c + 1] = it.wbase[c] + 32 * (int64_t)len;
        }
    }
    it.w.assign(2 * (size_t)it.wbase[NI], 0.0f);
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; j++) {
            const uint16_t* cnt = &rows.cnt[(size_t)j * nm];
            int64_t ns = rows.src_off[j + 1] - rows.src_off[j];
            std::vector<int64_t> off(nm + 1, 0);
            for (int i = 0; i < nm; i++) off[i + 1] = off[i] + cnt[i];
            for (int64_t c = it.item_ptr[j]; c < it.item_ptr[j + 1]; c++) {
                int r0 = (int)(32 * (c - it.item_ptr[j]));
                for (int l = 0; l < 32; l++)
                    if (r0 + l < ns) it.src[c * 32 + l] = rows.src[rows.src_off[j] + r0 + l];
                // slice by slice, lanes innermost: both the row's m-major weights and the item's
                // element pairs are read and written contiguously
                for (int t = 0; t < it.len[c]; t++) {
                    int i = it.s0[c] + t;
                    if (i >= nm) continue;
                    const int lanes = std::min<int64_t>(32, std::min<int64_t>(ns, (int64_t)cnt[i]) - r0);
                    for (int l = 0; l < lanes; l++) {
                        int64_t from = 2 * (rows.w_off[j] + off[i] + r0 + l);
                        int64_t to = 2 * (it.wbase[c] + 64 * (int64_t)(t >> 1) + 2 * l + (t & 1));
                        it.w[to] = rows.w[from];
                        it.w[to + 1] = rows.w[from + 1];
                    }
                }
            }
        }
    });
    return WAVE1D_OK;
}

int build_receivers(HostPlan& hp, const double* xr, int64_t R, std::string& err) {
    const Params& P = hp.P;
    hp.P.R = R;
    hp.xr.assign(xr, xr + R);
    double omega_lim = kPi - 3.0 * std::max(P.delta, P.delta_s);
    for (int64_t r = 0; r < R; r++) {
        double v = hp.xr[r];
        if (!std::isfinite(v)) { err = "non-finite receiver position"; return WAVE1D_EINVAL; }
        if (P.bc == WAVE1D_PERIODIC) {
            v = std::fmod(v + kPi, 2.0 * kPi);
            if (v < 0) v += 2.0 * kPi;
            v -= kPi;
            if (v >= kPi) v -= 2.0 * kPi;
        } else if (std::fabs(v) > omega_lim) {
            err = "free-space receiver outside Omega (Sec. 4.4)";
            return WAVE1D_EDOMAIN;
        }
        hp.xr[r] = v;
    }
    if (hp.range) {
        // the receivers' local part is summed over index windows (sources within delta)
        const int64_t M = P.M;
        const bool per = P.bc == WAVE1D_PERIODIC;
        const int64_t elo = per ? -M : 0, ehi = per ? 2 * M : M;
        const double reach = P.delta * (1.0 + 1e-12) + 1e-13;
        hp.r_win.assign(2 * (size_t)R, 0);
        for (int64_t r = 0; r < R; r++) {
            const double xv = hp.xr[r];
            hp.r_win[2 * r] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(hp.x, M, e) > xv - reach; });
            hp.r_win[2 * r + 1] = (int32_t)first_true(elo, ehi, [&](int64_t e) { return x_ext(hp.x, M, e) >= xv + reach; });
        }
        spread_weights(P, hp.xr, hp.rc_i0, hp.rc_ker);
        return WAVE1D_OK;
    }
    Window win(P.delta, P.b);
    int rc = build_local(P, win, hp.xr, hp.x, true, hp.rloc, nullptr, INT64_MAX, err);
    if (rc) return rc;
    // m >= 1 terms go to the item layout (summed concurrently with the history part); the m = 0
    // terms of sources closer than dt need sigma^{n+1} and are kept as a short list
    if ((rc = build_rows(hp.rloc, 1, hp.rrows, err))) return rc;
    build_items(hp.rrows, hp.ritems);
    hp.r0_ptr.assign(R + 1, 0);
    hp.r0_src.clear();
    hp.r0_w.clear();
    for (int64_t r = 0; r < R; r++) {
        for (int64_t q = hp.rloc.row_ptr[r]; q < hp.rloc.row_ptr[r + 1]; q++) {
            int lo = hp.rloc.mrange[q] & 0xffff, cnt = hp.rloc.mrange[q] >> 16;
            if (lo == 0 && cnt > 0) {
                hp.r0_src.push_back(hp.rloc.src[q]);
                hp.r0_w.push_back(hp.rloc.w[hp.rloc.woff[q]]);
            }
        }
        hp.r0_ptr[r + 1] = (int64_t)hp.r0_src.size();
    }
    spread_weights(P, hp.xr, hp.rc_i0, hp.rc_ker);
    return WAVE1D_OK;
}

void local_weights_exact(const Params& P, const std::vector<double>& d, std::vector<double>& Q) {
    Window win(P.delta, P.b);
    LocalRule rule;
    rule.init(P, win);
    const int nm = P.m_max + 1;
    Q.assign(d.size() * (size_t)nm, 0.0);
    for (size_t i = 0; i < d.size(); i++) rule.weights(d[i], &Q[i * nm]);
}

// Breakpoints of the local rule (Sec. 4.1): node i of the N_L-point Gauss-Legendre rule over
// [d, delta] sits at s = d + (delta - d) c_i, c_i = (x_i + 1) / 2, and switches its p-point stencil
// where s crosses a multiple of dt; d = dt switches m_min.  Breakpoints closer than 1e-9 dt are
// merged (the kink between them moves a weight by at most ~1e-11 of its size, for distances
// within 1e-9 dt of it); dt itself is kept exactly.  On every interval each Q_m (m = 0 .. m_max)
// is interpolated at the 8 Chebyshev points of the first kind of z = (d - mid) ih, where ih =
// fl32(1 / half-width) is the scale the device uses, then written in monomials of z.
constexpr double kRangeMaxWidth = 0.15;

void build_range_tables(const Params& P, RangeTables& rt) {
    rt = RangeTables();
    rt.nm = P.m_max + 1;
    std::vector<double> gx, gw;
    gauss_legendre(P.NL, gx, gw);
    std::vector<double> cand = {P.dt};
    for (double xg : gx) {
        const double c = 0.5 * (xg + 1.0);
        for (int k = 0; k <= P.W + 1; k++) {
            const double d = ((double)k * P.dt - P.delta * c) / (1.0 - c);
            if (d > 0.0 && d < P.delta) cand.push_back(d);
        }
    }
    std::sort(cand.begin(), cand.end());
    const double gap = 1e-9 * P.dt;
    rt.bp.push_back(0.0);
    for (double v : cand) {
        if (std::fabs(v - P.dt) <= gap && v != P.dt) continue;       // dt stays exact
        if (v - rt.bp.back() <= gap) {
            if (v == P.dt) rt.bp.back() = P.dt;                       // replace a neighbour by dt
            continue;
        }
        if (P.delta - v <= gap) continue;
        rt.bp.push_back(v);
    }
    rt.bp.push_back(P.delta);
    {
        // intervals wider than kRangeMaxWidth dt are cut into equal parts: the curvature
        // coefficients (single floats on the device) shrink with the width as width^r
        const char* env = std::getenv("WAVE1D_RANGE_WIDTH");
        const double cap = (env ? std::atof(env) : kRangeMaxWidth) * P.dt;
        std::vector<double> cut = {rt.bp[0]};
        for (size_t i = 1; i < rt.bp.size(); i++) {
            const double a = rt.bp[i - 1], b = rt.bp[i];
            const int parts = (int)std::ceil((b - a) / cap - 1e-9);
            for (int q = 1; q < parts; q++) cut.push_back(a + (b - a) * q / parts);
            cut.push_back(b);
        }
        rt.bp.swap(cut);
    }
    rt.nint = (int)rt.bp.size() - 1;
    rt.iv_dt = (int)(std::find(rt.bp.begin(), rt.bp.end(), P.dt) - rt.bp.begin());
    rt.cell_scale = (float)(kRsCells / P.delta);
    rt.cell.assign(kRsCells, 0);
    for (int c = 0; c < kRsCells; c++) {
        const double d = (double)c / (double)rt.cell_scale;
        rt.cell[c] = std::max(0, std::min(rt.nint - 1, (int)(std::upper_bound(rt.bp.begin(), rt.bp.end(), d) - rt.bp.begin()) - 1));
    }
    const int n = rt.nint, nm = rt.nm, np = 8;
    rt.bp2.resize(2 * (size_t)(n + 1));
    for (int i = 0; i <= n; i++) {
        const float h = (float)rt.bp[i];
        rt.bp2[2 * i] = h;
        rt.bp2[2 * i + 1] = (float)(rt.bp[i] - (double)h);
    }
    rt.mid.resize(n);
    rt.ih.resize(n);
    std::vector<double> dn((size_t)n * np);
    double zk[np];
    for (int k = 0; k < np; k++) zk[k] = std::cos(kPi * (k + 0.5) / np);
    for (int iv = 0; iv < n; iv++) {
        const double a = rt.bp[iv], b = rt.bp[iv + 1], mid = 0.5 * (a + b);
        // the reference point of the interval's polynomials (the midpoint to 48 bits)
        const float mh = (float)mid, ml = (float)(mid - (double)mh);
        rt.mid[iv] = (double)mh + (double)ml;
        rt.ih[iv] = (float)(2.0 / (b - a));
        for (int k = 0; k < np; k++) dn[(size_t)iv * np + k] = rt.mid[iv] + zk[k] / (double)rt.ih[iv];
    }
    std::vector<double> Q;
    local_weights_exact(P, dn, Q);
    // Chebyshev coefficients, then monomials: T_{r+1} = 2 z T_r - T_{r-1}
    double T[np][np] = {};
    T[0][0] = 1.0;
    T[1][1] = 1.0;
    for (int r = 1; r + 1 < np; r++)
        for (int q = 0; q < np; q++) T[r + 1][q] = (q > 0 ? 2.0 * T[r][q - 1] : 0.0) - T[r - 1][q];
    rt.cheb.assign((size_t)n * nm * np, 0.0);
    rt.coef.assign((size_t)n * nm * 12, 0.0f);
    rt.mr.assign(2 * (size_t)n, 0);
    rt.mr0.assign(2 * (size_t)n, 0);
    for (int iv = 0; iv < n; iv++) {
        int lo = nm, hi = -1, lo1 = nm, hi1 = -1;
        for (int m = 0; m < nm; m++) {
            double c[np], a[np];
            bool nz = false;
            for (int r = 0; r < np; r++) {
                double sum = 0.0;
                for (int k = 0; k < np; k++) sum += Q[((size_t)iv * np + k) * nm + m] * std::cos(kPi * r * (k + 0.5) / np);
                c[r] = sum * (r == 0 ? 1.0 : 2.0) / np;
                nz = nz || c[r] != 0.0;
            }
            for (int q = 0; q < np; q++) {
                a[q] = 0.0;
                for (int r = q; r < np; r++) a[q] += c[r] * T[r][q];
            }
            double* cd = &rt.cheb[((size_t)iv * nm + m) * np];
            for (int r = 0; r < np; r++) cd[r] = c[r];
            float* cf = &rt.coef[((size_t)iv * nm + m) * 12];
            for (int q = 0; q < 4; q++) {
                const float h = (float)a[q];
                cf[2 * q] = h;
                cf[2 * q + 1] = (float)(a[q] - (double)h);
            }
            for (int q = 4; q < np; q++) cf[4 + q] = (float)a[q];
            if (nz) {
                lo = std::min(lo, m);
                hi = std::max(hi, m);
                if (m >= 1) {
                    lo1 = std::min(lo1, m);
                    hi1 = std::max(hi1, m);
                }
            }
        }
        rt.mr0[2 * iv] = lo;
        rt.mr0[2 * iv + 1] = hi;
        rt.mr[2 * iv] = lo1;
        rt.mr[2 * iv + 1] = hi1;
    }
}

void receiver_columns(const LocalCSR& rloc, int64_t M, ReceiverColumns& out) {
    const int64_t R = rloc.row_ptr.empty() ? 0 : (int64_t)rloc.row_ptr.size() - 1;
    const int64_t n = R > 0 ? rloc.row_ptr[R] : 0;
    out.src_ptr.assign(M + 1, 0);
    for (int64_t e = 0; e < n; e++) out.src_ptr[rloc.src[e] + 1]++;
    for (int64_t l = 0; l < M; l++) out.src_ptr[l + 1] += out.src_ptr[l];
    out.rcv.assign(n, 0);
    out.mrange.assign(n, 0);
    out.woff.assign(n, 0);
    std::vector<int64_t> fill(out.src_ptr.begin(), out.src_ptr.end() - 1);
    for (int64_t r = 0; r < R; r++)                  // receivers in order: each source's list ascends in r
        for (int64_t e = rloc.row_ptr[r]; e < rloc.row_ptr[r + 1]; e++) {
            const int64_t f = fill[rloc.src[e]]++;
            out.rcv[f] = (int32_t)r;
            out.mrange[f] = rloc.mrange[e];
            out.woff[f] = rloc.woff[e];
        }
}

}  // namespace wave1d
