// Reads "M dt delta" and M positions from standard input; prints the largest block of springs
// closer than dt and the ordered pairs closer than delta that the batched plan's form rule uses
// (instance_shape, csrc/batch_host.cpp).
#include <cstdio>
#include <vector>

#include "batch_host.h"

int main() {
    long long M;
    double dt, delta;
    if (std::scanf("%lld %lf %lf", &M, &dt, &delta) != 3) return 2;
    std::vector<double> x((size_t)M);
    for (long long j = 0; j < M; j++)
        if (std::scanf("%lf", &x[j]) != 1) return 2;
    const wave1d::InstanceShape s = wave1d::instance_shape(x.data(), M, dt, delta);
    std::printf("%lld %lld\n", (long long)s.largest_block, (long long)s.pairs);
    return 0;
}
