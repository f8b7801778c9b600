// Host-side check (no GPU) of the piecewise-polynomial local weights (local_fit.h) against the
// plan's own rule: input dt tol p deg nsamples; builds a one-spring plan for the parameters, the
// fit, and compares Q_m(d) at nsamples pseudo-random distances in [0, delta) plus every breakpoint
// midpoint.  Prints "ok <intervals> <table doubles> <max |error| / max |Q|>".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "internal.h"
#include "local_fit.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    double dt, tol;
    int p, deg, ns;
    if (std::scanf("%lf %lf %d %d %d", &dt, &tol, &p, &deg, &ns) != 5) return 2;
    double x = 0.0, beta = 1.0;
    HostPlan hp;
    std::string err;
    if (build_host_plan(&x, &beta, 1, WAVE1D_PERIODIC, dt, 10, tol, p, 0.5, 0, 0, 32, 0, 0, 4096, (int64_t)1 << 30, hp,
                        err)) {
        std::printf("error %s\n", err.c_str());
        return 1;
    }
    const Params& P = hp.P;
    LocalFit f;
    build_local_fit(P, deg, f);
    std::vector<double> d;
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> u(0.0, P.delta);
    for (int i = 0; i < ns; i++) d.push_back(u(g));
    for (size_t i = 0; i + 1 < f.bp.size(); i++) d.push_back(0.5 * (f.bp[i] + f.bp[i + 1]));
    std::vector<double> Q;
    local_weights_exact(P, d, Q);
    const int nm = P.m_max + 1;
    double scale = 0.0, worst = 0.0;
    std::vector<double> q(nm);
    for (size_t i = 0; i < d.size(); i++) {
        local_fit_eval(f, d[i], q.data());
        for (int m = 0; m < nm; m++) {
            scale = std::max(scale, std::fabs(Q[i * nm + m]));
            worst = std::max(worst, std::fabs(q[m] - Q[i * nm + m]));
        }
    }
    std::printf("ok %zu %zu %.3e\n", f.bp.size() - 1, f.coef.size(), worst / scale);
    return 0;
}
