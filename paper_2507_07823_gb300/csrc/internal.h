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

// The same weights regrouped for the step kernel (Sec. 4.1 local sum), one row per target:
// sources sorted by the first m they need (m_lo, which grows with the distance), and for each
// m = m_first .. m_top the weights of the cnt[m] sources active at that m (a prefix of the sorted
// list), stored m-major so a warp reads each m's weights contiguously.  Weights are split into a
// pair of floats (hi = fl(Q), lo = fl(Q - hi)) for compensated FP32 arithmetic.
struct LocalRows {
    int m_first = 1, nm = 0;            // m = m_first .. m_first + nm - 1
    std::vector<int64_t> src_off;       // rows + 1
    std::vector<int32_t> src;           // per row, sorted sources
    std::vector<int64_t> w_off;         // rows + 1 (in weights)
    std::vector<uint16_t> cnt;          // rows * nm
    std::vector<float> w;               // 2 floats per weight (hi, lo)
};

// The local weights as independent work items of 32 sources (a "chunk" of one target row): lane l
// of item c handles source rank 32 c + l of its row and walks the m-slices s0 .. s0 + len - 1; the
// weights of elements 2u, 2u+1 are at w[wbase + 64 u + 2 l + {0, 1}] (zero before the source's
// first slice, past the row's last source, and in the padding that makes len even), so a warp reads
// one contiguous 512-byte line per element pair.
struct LocalItems {
    int m_first = 1;
    std::vector<int64_t> item_ptr;      // rows + 1
    std::vector<int32_t> row;           // per item
    std::vector<int32_t> s0, len;       // first slice, number of slices
    std::vector<int64_t> wbase;         // offset (in weights) of element 0, lane 0
    std::vector<int32_t> src;           // 32 per item (source index, 0 for padded lanes)
    std::vector<float> w;               // 2 floats per weight (hi, lo)
};
int build_items(const LocalRows& rows, LocalItems& items);

// Local weights as polynomials of the pair distance (plans opened with opts.local_weights = 1,
// which hold no per-pair data).  Q_m(d) is smooth between the breakpoints of the Gauss-Legendre
// rule (a node crossing a multiple of dt, and d = dt, Sec. 4.1); on interval iv it is a degree-7
// polynomial of z = (d - mid_iv) ih_iv with ih_iv = fl32(1 / half-width): the device computes z
// with that single-precision scale, and the series are fitted for exactly that map.
struct RangeTables {
    int nint = 0, nm = 0, iv_dt = 0;   // intervals, m = 0 .. nm - 1, index of the breakpoint dt
    std::vector<double> bp;            // nint + 1 breakpoints, bp[0] = 0, bp[iv_dt] = dt, bp[nint] = delta
    std::vector<float> bp2;            // the same as (hi, lo) pairs
    std::vector<double> mid;           // per interval: midpoint (rounded to a float pair's 48 bits)
    std::vector<float> ih;             // per interval: fl32(1 / half-width)
    std::vector<int32_t> mr;           // per interval: first and last m >= 1 with a non-zero series
    std::vector<int32_t> mr0;          // per interval: first and last m >= 0 with a non-zero series
    std::vector<float> coef;           // [iv][m][12]: monomial coefficients of z, a0 .. a3 as (hi, lo)
                                       //   pairs, a4 .. a7 single
    std::vector<double> cheb;          // [iv][m][8]: Chebyshev coefficients in z (FP64)
    std::vector<int32_t> cell;         // kRsCells: interval of the left end of each cell of [0, delta)
    float cell_scale = 0.f;            // kRsCells / delta: cell of a distance d is floor(d cell_scale)
};
void build_range_tables(const Params& P, RangeTables& out);
// The plan's weight rule itself at each distance, Q[i * (m_max + 1) + m] (for checks).
void local_weights_exact(const Params& P, const std::vector<double>& d, std::vector<double>& Q);
// targets per block of the range-mode local sum (one per thread); cells of the distance lookup table
constexpr int kRsTargets = 256;
constexpr int kRsTTargets = 128;    // outputs per block of the transposed local sum (reverse march)
constexpr int kRsCells = 2048;

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
    std::vector<double> modefac;       // [k][8]: deconv1, Re/Im deconv1 e^{2 pi i k/nf},
                                       //         Re/Im deconv2 (1 + i e^{-2 pi i k/nf}),
                                       //         Re/Im deconv2 (1 - i e^{-2 pi i (L-k)/nf}), 0
    std::vector<double> tw2K;          // [a][2] e^{i pi a / K}, a < 2K (radiation projection)
    std::vector<int32_t> g_ptr;        // nf + 1: spreading as a sparse matrix, rows in column-pass
                                       //   order 2 (i2 L1 + i1) + h
    std::vector<int32_t> g_src;        //   spring of each entry (internal order)
    std::vector<double> g_w;           //   kernel weight of each entry
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
    LocalRows lrows;                   // springs, m-major rows
    LocalRows rrows;                   // receivers, m-major rows
    LocalItems litems;                 // springs, step-kernel layout
    LocalItems ritems;                 // receivers, m >= 1, step-kernel layout
    std::vector<int64_t> r0_ptr;       // receivers: sources closer than dt with their m = 0 weight
    std::vector<int32_t> r0_src;
    std::vector<double> r0_w;
    // implicit blocks of I + S (eq. linearSystem), inverted
    std::vector<int64_t> blk_ptr;      // blocks + 1 into blk_members
    std::vector<int32_t> blk_members;  // internal spring indices
    std::vector<int64_t> blk_inv_off;  // offset of each block's inverse in inv
    std::vector<double> inv;           // column-major inverses: inv[l * s + i] = inverse[i][l]
    int64_t max_block = 0;
    // solve groups: consecutive blocks of at most 32 members packed into the 32 lanes of a warp
    std::vector<int32_t> sg_j;         // [group][32]: spring of the lane, -1 for an idle lane
    std::vector<int32_t> sg_meta;      // [group][32]: first lane of the lane's block | size << 8 |
                                       //   row in the block << 16
    std::vector<int64_t> sg_off;       // [group][32]: offset of the lane's block inverse in inv
    std::vector<double> sg_beta;       // [group][32]: stiffness of the lane's spring
    std::vector<int64_t> sg_ip;        // [group][32]: first local-sum item of the lane's row
    std::vector<int32_t> sg_icnt;      // [group][32]: its number of items
    std::vector<int32_t> sg_smax;      // [group]: largest block of the group
    std::vector<int64_t> big_blk;      // blocks of more than 32 members, one entry per 32 rows
    std::vector<int32_t> big_row0;     //   (a single entry above 256 members): first row
    // no pair lists (opts.local_weights = 1): the weights as polynomials of the distance, the
    // positions as (hi, lo) float pairs, and index windows into the sorted springs.  Windows are
    // "extended" indices e in [-M, 2M) in the periodic box (spring e mod M shifted by
    // 2 pi floor(e / M)), in [0, M) in free space.
    bool range = false;
    RangeTables rt;
    std::vector<int32_t> nb_lo, nb_cnt;// springs: window of the sources closer than dt (FP64 test
                                       //   |x_e - x_j| < dt), the implicit part of eq. linearSystem
    std::vector<int64_t> nb_off;       // M + 1: offsets of their weights
    std::vector<int32_t> blk_win;      // per block of kRsTargets targets: first source of the delta
                                       //   window, first source at or right of the first target,
                                       //   first source right of the last target, end of the window
    std::vector<int32_t> r_win;        // receivers: [lo, hi) window of sources within delta
    int64_t range_pairs = 0;           // (target, source) pairs closer than delta (springs)
    // radiation projection: grid points i of the 2K-point grid that are rolled off
    std::vector<int32_t> rbc_idx;      // 4W grid indices
    std::vector<double> rbc_x;         // their positions
    std::vector<double> rbc_phi;       // phi_s(arg), arg = pi - delta_s -/+ x
    std::vector<double> rbc_dphi;      // phi_s'(arg)
};

// Dynamic shared memory of k_fft_cols / k_fft_rows for a line of N points: the line itself and
// its N/2 twiddles (every launch site must use this).
inline size_t fft_smem_bytes(int N) { return (size_t)(N + N / 2) * 16; }
// threads of a block of the one-launch step kernel
constexpr int kStepThreads = 256;

// window width in steps: W given, else ceil(2 ln(1/tol) / (pi gamma)) (eqs. b, W)
int window_steps(double tol, double gamma, int W);
// Returns 0 or a negative wave1d_status; fills err with a message on failure.
int build_host_plan(const double* x, const double* beta, int64_t M, int bc, double dt, int64_t Nt,
                    double tol, int p, double gamma, int W, int NL, int Ng, int nufft_w,
                    int rbc_period, int max_block, int64_t max_local_bytes, HostPlan& hp,
                    std::string& err, bool range = false);
int build_receivers(HostPlan& hp, const double* xr, int64_t R, std::string& err);
int build_rows(const LocalCSR& csr, int m_first, LocalRows& rows, std::string& err);

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
    double* ftail;            // [K+1][4]: FIR tail (taps m >= 1) of h_k, g_k of the step
    double* alpha;            // [K+1][2]
    double* alpha_p;          // [K+1][2]
    // NUFFT buffers
    double* grid;             // nf reals (forward input / inverse output)
    double* spec;             // L complex, forward FFT output
    double* spec2;            // L complex, type-2 spectrum (inverse FFT input; zero outside |k| <= K)
    double* work;             // L complex (between FFT stages)
    double* rhs;              // M, right-hand sides of the block solve (internal order)
    double* gforce;           // M, forcing g_j(t_{n+1}) computed ahead by the step kernel
    const int32_t* sp_i0;
    const double* sp_ker;
    const int32_t* rc_i0;
    const double* rc_ker;
    double* uH;               // M (internal order)
    double* uHr;              // R
    double* clocal;           // M, local explicit sum of the step
    // density rings, time-major: sig[(q mod ring) * M + j] = sigma_j^q, and the same values as
    // float pairs (hi, lo) in sig2 for the compensated local sum
    double* sig;
    float* sig2;              // interleaved (hi, lo)
    // local part, step-kernel layout (see LocalItems); sig2 holds 2 * ring slots (slot s and s + ring
    // carry the same values) so a walk over m never wraps
    int l_mfirst, r_mfirst;
    int64_t l_nitems, r_nitems;
    const int64_t* l_item_ptr;
    const int32_t* l_row;
    const int32_t* l_s0;
    const int32_t* l_len;
    const int64_t* l_wbase;
    const int32_t* l_src;
    const float* l_w;             // interleaved (hi, lo)
    const int64_t* r_item_ptr;
    const int32_t* r_s0;
    const int32_t* r_len;
    const int64_t* r_wbase;
    const int32_t* r_src;
    const float* r_w;
    double* l_part;               // per spring item: partial local sum
    double* r_part;               // per receiver item: partial local sum (m >= 1)
    unsigned long long* item_ctr; // items handed out in this step (reset once they are done)
    const int32_t* item_order;    // spring then receiver items (o >= l_nitems: receiver item
                                  //   o - l_nitems), longest first
    int r0_stride;                // receivers: m = 0 terms (sources closer than dt), padded to
    const int32_t* r0p_src;       //   r0_stride entries per receiver (zero weight on padding)
    const double* r0p_w;
    // spreading matrix and per-mode factors
    const int32_t* g_ptr;
    const int32_t* g_src;
    const double* g_w;
    const double* modefac;
    const double* tw2K;
    // blocks
    const int64_t* blk_ptr;
    const int32_t* blk_members;
    const int64_t* blk_inv_off;
    const int32_t* sg_j;
    const int32_t* sg_meta;
    const int64_t* sg_off;
    const double* sg_beta;
    const int64_t* sg_ip;
    const int32_t* sg_icnt;
    const int32_t* sg_smax;
    const int64_t* big_blk;
    const int32_t* big_row0;
    int64_t n_sgroups, n_big;
    const double* inv;
    int64_t nblocks, inv_len;
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
    // receivers' positions (device copy)
    const double* xr;
    // one-launch step kernel: blocks [0, hist_blocks) start with the history pipeline;
    // bar[0..15] are its work and barrier counters (zero between steps)
    int hist_blocks;
    unsigned* bar;
    unsigned spin_limit;      // polls before a wait gives up (WAVE1D_ETIMEOUT)
    int hold_unit;            // test hook: 1 = the first column unit is never counted
};

// Device view of the range-mode tables (plans opened with opts.local_weights = 1), passed by value
// beside DevPlan.
struct RangeDev {
    int nint, nm, iv_dt, nblk;
    double delta;
    const float* bp2;           // nint + 1 breakpoints (hi, lo)
    const float* ih;            // nint scales
    const int32_t* mr;          // nint x 2: m range of the local sum (m >= 1)
    const int32_t* mr0;         // nint x 2: m range with m = 0
    const float* coef;          // [iv][m][12]: a0 .. a3 as (hi, lo) pairs, a4 .. a7
    const double* bp;           // nint + 1 breakpoints (FP64)
    const double* mid;          // nint midpoints
    const double* cheb;         // [iv][m][8] Chebyshev coefficients in z (FP64)
    const int* cell;            // kRsCells: first interval of each cell of [0, delta)
    float cell_scale;           // kRsCells / delta
    const int32_t* blk_win;     // [block][4] (see HostPlan::blk_win)
    const int32_t* nb_lo;       // M
    const int32_t* nb_cnt;      // M
    const int64_t* nb_off;      // M + 1
    float* nb_w;                // (beta_j / 2) Q_0(d_jl) as (hi, lo), the entry l = j zero
    double* diag;               // M: 1 + (beta_j / 2) Q_0(0)
    double* it64[2];            // Jacobi iterates (FP64) and the same as (hi, lo) pairs
    float* it2[2];
    unsigned long long* stats;  // [kRsMaxIter + 1][2]: max |change|, max |sigma| of each iterate (bits)
    int* iters;                 // Jacobi sweeps of the last step
    const int32_t* r_win;       // [R][2]
    double* r_part;             // [R][rchunks]: receivers' local sums by source chunk
    int rchunks;
};
// Jacobi sweeps of the implicit solve at most, and the stopping rule: max |change| <=
// kRsTol max |sigma| (the sweeps contract by max_j sum_l |S_jl| / (1 + S_jj), about 0.14 for a
// million clustered springs at dt = 5e-4)
constexpr int kRsMaxIter = 40;
constexpr double kRsTol = 1e-14;

}  // namespace wave1d
