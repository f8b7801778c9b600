// Reads "n_inst dt tol local_weights max_block max_local_bytes", then per instance "M" and M
// positions; runs the batched plan's split of instances by form (batch_instances,
// csrc/batch_host.cpp) with stiffnesses 3 and no receivers, and prints
//   "forms f_0 .. f_{n-1}" and, per joined instance, "joined b nw8 padded" (its stored weights at
//   8 bytes each, the budget's measure, and the bytes its work items take), or "error rc message".
#include <cstdio>
#include <cstring>
#include <vector>

#include "batch_host.h"

int main() {
    int n, lw, max_block;
    double dt, tol;
    long long max_bytes;
    if (std::scanf("%d %lf %lf %d %d %lld", &n, &dt, &tol, &lw, &max_block, &max_bytes) != 6) return 2;
    std::vector<int64_t> off(1, 0);
    std::vector<double> x;
    for (int b = 0; b < n; b++) {
        long long M;
        if (std::scanf("%lld", &M) != 1) return 2;
        for (long long j = 0; j < M; j++) {
            double v;
            if (std::scanf("%lf", &v) != 1) return 2;
            x.push_back(v);
        }
        off.push_back(off.back() + M);
    }
    std::vector<double> beta(x.size(), 3.0);
    wave1d_opts o;                          // wave1d_opts_default's values (that call lives in the CUDA library)
    std::memset(&o, 0, sizeof(o));
    o.p = 8;
    o.gamma = 0.5;
    o.Ng = 32;
    o.step_kernel = 1;
    o.local_weights = lw;
    o.max_block = max_block;
    o.max_local_bytes = max_bytes;
    std::vector<int> form, joined;
    std::vector<wave1d::HostPlan> inst;
    std::string err;
    const int rc = wave1d::batch_instances(n, off.data(), x.data(), beta.data(), nullptr, nullptr, dt, 10, tol, o, form,
                                           joined, inst, err);
    if (rc) {
        std::printf("error %d %s\n", rc, err.c_str());
        return 0;
    }
    std::printf("forms");
    for (int f : form) std::printf(" %d", f);
    std::printf("\n");
    for (size_t k = 0; k < joined.size(); k++)
        std::printf("joined %d %lld %lld\n", joined[k], (long long)inst[k].loc.woff.back() * 8,
                    (long long)inst[k].litems.w.size() * 4);
    return 0;
}
