// Internal layout of a wave1d plan: host-side tables built by plan_host.cpp and the device view
// the kernels read.  Springs are kept sorted by position inside the plan ("internal order").
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace wave1d {

// ---------------------------------------------------------------------------------------------
// Host tables (built once per plan, then copied to the device)
// ---------------------------------------------------------------------------------------------
struct Params {
    int64_t M = 0, R = 0, Nt = 0;
    int bc = 0;                 // 0 periodic, 1 free space
    double dt = 0, tol = 0, gamma = 0.5, b = 0, delta = 0;
    int K = 0, W = 0, m_max = 0, p = 8, NL = 0, Ng = 32;
    // NUFFT
    int nf = 0, L = 0, L1 = 0, L2 = 0, nufft_w = 0;
    double h_f = 0, kb_beta = 0;
    // radiation projection (free space)
    int rbc_period = 0;
    double h_rbc = 0, delta_s = 0;
    int ring = 0;               // slots of the density ring, m_max + 1
};

// Compressed sparse rows of local weights Q_m(d) for (target, source) pairs within delta.
struct LocalCSR {
    std::vector<int64_t> row_ptr;      // targets + 1
    std::vector<int32_t> src;          // source spring (internal order)
    std::vector<int32_t> mrange;       // m_lo | (m_cnt << 16)
    std::vector<int64_t> woff;         // offset of the pair's first weight in w
    std::vector<double> w;             // Q_m for m = m_lo .. m_lo + m_cnt - 1
    int64_t nearby = 0;                // pairs with d < dt
};

struct HostPlan {
    Params P;
    std::vector<int32_t> perm;         // internal index -> caller index
    std::vector<double> x, beta;       // internal order
    std::vector<double> xr;            // receivers (caller order == internal order)
    // history part
    std::vector<double> pq;            // [m][k][2] : dt p_k(m dt), dt q_k(m dt)
    std::vector<double> rot;           // [k][3]    : cos k dt, sin(k dt)/k, k sin k dt
    std::vector<double> deconv1;       // [k] type-1 deconvolution (-1)^k h / (2 pi psihat(k))
    std::vector<double> deconv2;       // [k] type-2 deconvolution (-1)^k h / psihat(k)
    std::vector<double> twiddle;       // [j][2] e^{+2 pi i j / L}, j < L
    // spreading / interpolation
    std::vector<int32_t> sp_i0;        // springs: first fine-grid index (wrapped)
    std::vector<double> sp_ker;        // springs: [j][w] kernel weights
    std::vector<int32_t> rc_i0;
    std::vector<double> rc_ker;
    std::vector<int32_t> bin_ptr;      // nf + 1: springs whose first grid index is c
    std::vector<int32_t> bin_list;     // internal spring indices grouped by bin
    // local part
    LocalCSR loc;                      // springs (m >= 1 only; m = 0 lives in the blocks)
    LocalCSR rloc;                     // receivers (m >= 0)
    // implicit blocks of I + S (eq. linearSystem), inverted
    std::vector<int64_t> blk_ptr;      // blocks + 1 into blk_members
    std::vector<int32_t> blk_members;  // internal spring indices
    std::vector<int64_t> blk_inv_off;  // offset of each block's inverse in inv
    std::vector<double> inv;           // row-major inverses
    int64_t max_block = 0;
    // radiation projection: grid points i of the 2K-point grid that are rolled off
    std::vector<int32_t> rbc_idx;      // 4W grid indices
    std::vector<double> rbc_x;         // their positions
    std::vector<double> rbc_phi;       // phi_s(arg), arg = pi - delta_s -/+ x
    std::vector<double> rbc_dphi;      // phi_s'(arg)
};

// Returns 0 or a negative wave1d_status; fills err with a message on failure.
int build_host_plan(const double* x, const double* beta, int64_t M, int bc, double dt, int64_t Nt,
                    double tol, int p, double gamma, int W, int NL, int Ng, int nufft_w,
                    int rbc_period, int max_block, int64_t max_local_bytes, HostPlan& hp,
                    std::string& err);
int build_receivers(HostPlan& hp, const double* xr, int64_t R, std::string& err);

// ---------------------------------------------------------------------------------------------
// Device view (passed by value to kernels)
// ---------------------------------------------------------------------------------------------
struct DevPlan {
    // sizes
    int64_t M, R;
    int K, W, m_max, ring, nf, L, L1, L2, w, bc, npulse;
    double dt;
    // step counter and status word
    int64_t* step;            // [0] = n (steps taken), [1] = blocks finished in the last kernel
    int* status;              // 0 ok, else a wave1d_status latched by a kernel
    // springs
    const double* x;
    const double* beta;
    const int32_t* perm;
    // incident pulses (device copies)
    const double* pulse;      // [i][3] amp, center, width
    const double* g_ext;      // external forcing for the next step (internal order) or null
    // history part
    const double* pq;
    const double* rot;
    const double* deconv1;
    const double* deconv2;
    const double* twiddle;
    double* Sring;            // [W][K+1][2]
    double* alpha;            // [K+1][2]
    double* alpha_p;          // [K+1][2]
    // NUFFT buffers
    double* grid;             // nf reals (forward input / inverse output)
    double* spec;             // L complex, forward FFT output
    double* spec2;            // L complex, type-2 spectrum (inverse FFT input; zero outside |k| <= K)
    double* work;             // L complex (between FFT stages)
    double* rhs;              // M, right-hand sides of the block solve (internal order)
    const int32_t* sp_i0;
    const double* sp_ker;
    const int32_t* rc_i0;
    const double* rc_ker;
    const int32_t* bin_ptr;
    const int32_t* bin_list;
    double* uH;               // M (internal order)
    double* uHr;              // R
    // local part
    const int64_t* row_ptr;
    const int32_t* src;
    const int32_t* mrange;
    const int64_t* woff;
    const double* wq;
    const int64_t* rrow_ptr;
    const int32_t* rsrc;
    const int32_t* rmrange;
    const int64_t* rwoff;
    const double* rwq;
    double* clocal;           // M
    // density ring, time-contiguous per spring: sig[j * ring + (q mod ring)] = sigma_j^q
    double* sig;
    // blocks
    const int64_t* blk_ptr;
    const int32_t* blk_members;
    const int64_t* blk_inv_off;
    const double* inv;
    int64_t nblocks;
    // outputs recorded per step (chunk history, caller order for sigma)
    double* rec_hist;         // [chunk][R]
    double* sig_hist;         // [chunk][M] or null
    int chunk;
    // radiation projection
    const int32_t* rbc_idx;
    const double* rbc_x;
    const double* rbc_phi;
    const double* rbc_dphi;
    double* rbc_uv;           // [4W][4] : u, v before; du, dv
    double rbc_h;
};

}  // namespace wave1d
