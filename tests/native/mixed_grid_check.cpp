// Host-side check (no GPU) of the mixed-precision time step's premise: a time-step plan built with
// NUFFT width 7 and the standalone NUFFT plan at tol 1e-6 (which the mixed step runs on the plan's
// springs) have the same fine grid, FFT split, kernel shape, per-spring first cells and kernel
// values, and deconvolution factors, bit for bit.  Input: M dt tol bc p, then M positions and M
// stiffnesses.  Prints "ok" or the first difference.
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "nufft_host.h"
#include "wave1d.h"

using namespace wave1d;

int main() {
    long M;
    double dt, tol;
    int bc, p;
    if (std::scanf("%ld %lf %lf %d %d", &M, &dt, &tol, &bc, &p) != 5) return 2;
    std::vector<double> x(M), beta(M);
    for (auto& v : x) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : beta) if (std::scanf("%lf", &v) != 1) return 2;
    HostPlan hp;
    std::string err;
    int rc = build_host_plan(x.data(), beta.data(), M, bc, dt, 100, tol, p, 0.5, 0, 0, 32, 7, 0, 4096,
                             (int64_t)1 << 34, hp, err);
    if (rc) { std::printf("error %d %s\n", rc, err.c_str()); return 1; }
    Params PN;
    nufft_grid(PN, hp.P.K, 1e-6, 0);
    const Params& P = hp.P;
    if (PN.nf != P.nf || PN.L != P.L || PN.L1 != P.L1 || PN.L2 != P.L2 || PN.nufft_w != P.nufft_w ||
        PN.h_f != P.h_f || PN.kb_beta != P.kb_beta) {
        std::printf("grid differs: nf %d/%d w %d/%d beta %.17g/%.17g\n", PN.nf, P.nf, PN.nufft_w, P.nufft_w,
                    PN.kb_beta, P.kb_beta);
        return 1;
    }
    std::vector<int32_t> i0;
    std::vector<double> ker;
    spread_weights(PN, hp.x, i0, ker);
    if (i0 != hp.sp_i0 || ker != hp.sp_ker) { std::printf("spreading weights differ\n"); return 1; }
    std::vector<double> d1, d2, mf;
    nufft_factors(PN, d1, d2, mf);
    if (mf != hp.modefac || d1 != hp.deconv1 || d2 != hp.deconv2) { std::printf("deconvolution differs\n"); return 1; }
    std::printf("ok %d %d\n", P.nf, P.nufft_w);
    return 0;
}
