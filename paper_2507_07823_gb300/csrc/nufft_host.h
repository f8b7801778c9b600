// Host-side pieces of the Kaiser-Bessel NUFFT shared by the time-step plan and the standalone
// NUFFT plan: fine-grid sizing, per-point kernel weights and the deconvolution factors (Sec. 3.1).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace wave1d {

// spreading weights of eq. KB: i0[j] = first grid cell of point j (mod nf), ker[j * w + t] the
// kernel's value at cell i0[j] + t
void spread_weights(const Params& P, const std::vector<double>& x, std::vector<int32_t>& i0,
                    std::vector<double>& ker);
// deconvolution and real-FFT factors per mode k = 0..K
void nufft_factors(const Params& P, std::vector<double>& deconv1, std::vector<double>& deconv2,
                   std::vector<double>& modefac);
// fine grid (nf = power of two >= 2 (2K + 1), at least 64), kernel width for tol (or w_in > 0)
// and Kaiser-Bessel shape
void nufft_grid(Params& P, int K, double tol, int w_in);

// A cell range of the spreading pass: one block writes grid reals c0 .. c0 + nc - 1 of one instance
// complete, from the points whose first cell lies in the range or in the w - 1 cells before it (the
// halo, wrapping round the periodic box).  Those points are staged as the slice [a0, a0 + na) of
// the sorted order followed by [b0, b0 + nb); the run table at roff (nc + w entries) gives, for each
// of the nc + w - 1 cells from c0 - w + 1 on, the offset of its first staged point, then the total.
struct NuRange {
    int32_t a0, na, b0, nb;
    int32_t c0, nc, roff, lg;      // c0 = instance x nf + cell; lg = log2 of the lanes per cell
};
// Cut every instance's grid into ranges: points are sorted by first cell i0 (instance-local, in
// [0, nf)) instance by instance, instance b holding points [offsets[b], offsets[b+1]).  A range has
// at most max_cells cells and, where one cell allows, at most max_points points counting its halo;
// a stretch of cells no point reaches is one range of at most empty_cells cells (na + nb = 0, no run
// table).  lg: the largest power of two of lanes per cell, at most 32, that serves all nc + w - 1
// cells with `threads` threads.
void nufft_ranges(const std::vector<int32_t>& i0, const int64_t* offsets, int n_inst, int nf, int w,
                  int max_cells, int max_points, int empty_cells, int threads, std::vector<NuRange>& ranges,
                  std::vector<int32_t>& runs);

}  // namespace wave1d
