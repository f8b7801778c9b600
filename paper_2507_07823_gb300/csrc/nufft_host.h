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

}  // namespace wave1d
