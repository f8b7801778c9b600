// The local weights Q_m(d) (Sec. 4.1) as piecewise polynomials of the pair distance d, for
// computing weights from distances where storing them per pair does not fit.  Q_m is the N_L-point
// Gauss-Legendre rule over [d, delta] of (1 - phi) times the p-point interpolant; as d moves, the
// rule's nodes move, and a node crossing a multiple of dt switches its stencil, as does d crossing
// dt (the near/far rule).  Between those breakpoints Q_m is smooth, so each interval carries a
// Chebyshev series per m.
#pragma once

#include <vector>

#include "internal.h"

namespace wave1d {

struct LocalFit {
    int deg = 0;                 // Chebyshev degree per interval and m
    int nm = 0;                  // m = 0 .. nm - 1 (m_max + 1)
    std::vector<double> bp;      // breakpoints 0 = bp[0] < ... < bp[n] = delta
    std::vector<double> coef;    // [interval][m][deg + 1]
    std::vector<int> mlo, mhi;   // per interval: the first and last m with a non-zero series
};

// Breakpoints of the plan's rule and degree-`deg` series on every interval (fitted at the
// interval's Chebyshev points of the first kind, which avoid the breakpoints themselves).
void build_local_fit(const Params& P, int deg, LocalFit& out);
// Q[0 .. nm-1] at distance d in [0, delta) from the series (zeros for d >= delta).
void local_fit_eval(const LocalFit& f, double d, double* Q);
// Real sources of every item of a LocalItems table built from `rows` (item c of a row holds the
// row's source ranks 32 c .. 32 c + 31, of which min(32, n - 32 c) exist).
void item_source_counts(const LocalRows& rows, const LocalItems& items, std::vector<int8_t>& nsrc);
// The plan's stored-weight rule itself at each distance, Q[i * (m_max + 1) + m] (for checks).
void local_weights_exact(const Params& P, const std::vector<double>& d, std::vector<double>& Q);

}  // namespace wave1d
