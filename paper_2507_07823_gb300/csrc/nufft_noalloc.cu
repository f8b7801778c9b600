// Type-1 NUFFT of device arrays that allocates no memory (wave1d_nufft1_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs under a device-memory budget reserved up
// front (a framework's caching allocator or a fixed arena), and code that must not trigger the
// implicit device-wide synchronisation that cudaMalloc / cudaFree can cause in the middle of a
// time-critical loop.  This entry point computes the same spectrum as the spreading + FFT stages
// of a plan, with every intermediate array (fine grid, FFT work buffers, twiddle table) in one
// file-scope __device__ array of fixed size.  Every GPU that loads the library holds that array
// (2 MiB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"
#include "../../include/wave1d.h"

namespace wave1d {
__global__ void k_fft_cols(const double2*, double2*, const double2*, int, int, int, int, int);
__global__ void k_fft_rows(const double2*, double2*, const double2*, int, int, int, int, int);
}  // namespace wave1d

namespace {

constexpr int kMaxNf = 65536;                      // largest fine grid: K <= 16383
constexpr int kMaxDevices = 64;
constexpr size_t kScratchDoubles = 4 * (size_t)kMaxNf;   // grid, work, spectrum, twiddles

// Shared by every call on a device; holds the previous call's contents between calls.
static __device__ __align__(256) double g_nufft1_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// device address of the scratch array for the current device (looked up once per device)
int scratch_for_device(int dev, double** out, std::string& err) {
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device ordinal out of range";
        return WAVE1D_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_nufft1_scratch);
        if (e != cudaSuccess || !ptr) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return WAVE1D_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = (double*)g_scratch_ptr[dev];
    return WAVE1D_OK;
}

__global__ void k_na_prepare(double* grid, double2* tw, int nf, int L) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        grid[i] = 0.0;
        if (i < L) {
            double s, c;
            sincospi(2.0 * (double)i / (double)L, &s, &c);
            tw[i] = make_double2(c, s);
        }
    }
}

// Kaiser-Bessel spreading of unordered points, w taps each, double atomics on the scratch grid
__global__ void k_na_spread(const double* __restrict__ x, const double* __restrict__ cval,
                            int64_t M, double* grid, int nf, int w, double beta, double h) {
    const double kPi = 3.14159265358979323846;
    double inv_i0b = 1.0 / cyl_bessel_i0(beta);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        double u = (x[j] + kPi) / h;
        int64_t first = (int64_t)ceil(u - 0.5 * w);
        double cj = cval[j];
        for (int t = 0; t < w; t++) {
            double z = (double)(first + t - u) * 2.0 / w;
            double r = 1.0 - z * z;
            if (r <= 0.0) continue;
            double psi = cyl_bessel_i0(beta * sqrt(r)) * inv_i0b;
            int64_t i = (first + t) % nf;
            if (i < 0) i += nf;
            atomicAdd(&grid[i], cj * psi);
        }
    }
}

// S_k = (-1)^k h / (2 pi psihat(k)) * F_k,  F_k = E_k + e^{2 pi i k / nf} O_k from the half FFT
__global__ void k_na_post(const double2* __restrict__ Z, double* S, int K, int L, int nf, int w,
                          double beta, double h) {
    const double kPi = 3.14159265358979323846;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > K) return;
    double2 zk = Z[k];
    double2 zm = Z[k == 0 ? 0 : L - k];
    double ex = 0.5 * (zk.x + zm.x), ey = 0.5 * (zk.y - zm.y);
    double dx = 0.5 * (zk.x - zm.x), dy = 0.5 * (zk.y + zm.y);
    double ox = dy, oy = -dx;
    double s, c;
    sincospi(2.0 * (double)k / (double)nf, &s, &c);
    double fx = ex + c * ox - s * oy, fy = ey + c * oy + s * ox;
    double om = 0.5 * k * w * h;
    double r = sqrt(beta * beta - om * om);
    double psihat = w * h * (r > 0.0 ? sinh(r) / r : 1.0) / cyl_bessel_i0(beta);
    double d1 = ((k & 1) ? -1.0 : 1.0) * h / (2.0 * kPi * psihat);
    S[2 * k] = d1 * fx;
    S[2 * k + 1] = d1 * fy;
}

int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

}  // namespace

extern "C" int wave1d_nufft1_noalloc(const double* x, const double* c, int64_t M, int K,
                                     double tol, double* S, void* stream) {
    const double kPi = 3.14159265358979323846;
    if ((M > 0 && (!x || !c)) || !S || M < 0 || K < 1 || !(tol > 0.0 && tol < 0.1))
        return WAVE1D_EINVAL;
    // fine grid, kernel and FFT split (L = L1 L2, L1 >= L2) as a plan chooses them for this K and
    // tol; the spreading's atomic additions make the last bits differ from call to call
    int64_t nf = 1;
    while (nf < 2 * (2 * (int64_t)K + 1)) nf <<= 1;
    if (nf < 64) nf = 64;
    if (nf > kMaxNf) return WAVE1D_EUNSUPPORTED;       // beyond the fixed scratch array
    int L = (int)(nf / 2);
    int lg = ilog2i(L);
    int L1 = 1 << ((lg + 1) / 2), L2 = L / L1;
    int w = (int)std::ceil(std::log10(1.0 / tol)) + 1;
    w = w < 4 ? 4 : (w > 16 ? 16 : w);
    double upsamp = (double)nf / (2.0 * K + 1.0);
    double beta = kPi * w * (1.0 - 1.0 / (2.0 * upsamp));
    double h = 2.0 * kPi / (double)nf;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WAVE1D_ECUDA;
    double* base = nullptr;
    std::string err;
    int rc = scratch_for_device(dev, &base, err);
    if (rc != WAVE1D_OK) return rc;
    double* grid = base;                                   // nf reals
    double2* work = (double2*)(base + kMaxNf);             // L complex
    double2* spec = (double2*)(base + 2 * (size_t)kMaxNf); // L complex
    double2* tw = (double2*)(base + 3 * (size_t)kMaxNf);   // L complex
    cudaStream_t s = (cudaStream_t)stream;
    k_na_prepare<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(grid, tw, (int)nf, L);
    if (M > 0) {
        unsigned nb = (unsigned)std::min<int64_t>((M + 255) / 256, 4096);
        k_na_spread<<<nb, 256, 0, s>>>(x, c, M, grid, (int)nf, w, beta, h);
    }
    int t1 = L1 / 2 < 32 ? 32 : (L1 / 2 > 512 ? 512 : L1 / 2);
    int t2 = L2 / 2 < 32 ? 32 : (L2 / 2 > 512 ? 512 : L2 / 2);
    wave1d::k_fft_cols<<<L2, t1, wave1d::fft_smem_bytes(L1), s>>>((const double2*)grid, work, tw, L, L1,
                                                                  L2, ilog2i(L1), +1);
    wave1d::k_fft_rows<<<L1, t2, wave1d::fft_smem_bytes(L2), s>>>(work, spec, tw, L, L1, L2, ilog2i(L2),
                                                                  +1);
    k_na_post<<<(unsigned)((K + 1 + 127) / 128), 128, 0, s>>>(spec, S, K, L, (int)nf, w, beta, h);
    return cudaGetLastError() == cudaSuccess ? WAVE1D_OK : WAVE1D_ECUDA;
}
