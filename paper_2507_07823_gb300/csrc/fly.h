// Device view of the tables of the local sum with weights computed per pair (fly.cu).
#pragma once

#include <cstdint>

namespace wave1d {

struct FlyTables {
    const double* bp;        // nint + 1 breakpoints of the weight series (local_fit.h)
    const double* coef;      // [interval][m][deg + 1]
    const int* mlo;          // per interval: non-zero m range
    const int* mhi;
    int nint, deg, nm;
    const int8_t* l_nsrc;    // real sources of each spring item (1 .. 32)
    const int8_t* r_nsrc;    // real sources of each receiver item
    const double* xr;        // receiver positions
};

}  // namespace wave1d
