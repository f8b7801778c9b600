/*
 * wave1d — windowed Fourier projection (WFP) time marching for 1D waves scattered by point
 * springs, on one NVIDIA GB300 GPU (sm_103a).
 *
 * The method (arXiv 2507.07823): M springs of stiffness beta_j at x_j on a string, driven by an
 * incident wave u_inc(x, t) = f(x - t) (Sec. 1, eqs. uinc-gj).  The scattered field is the single
 * layer potential u = 1/2 sum_j int_0^{t - |x - x_j|} sigma_j (eq. singleLayerSol) whose
 * densities solve a Volterra system (eq. IEfree; eq. periodicIE in the periodic box [-pi, pi]).
 * Each time step splits the potential with a Kaiser-Bessel blending window of width
 * delta = W dt (eq. phi) into
 *   - a local part over the last delta of history, summed directly with Gauss-Legendre
 *     quadrature of p-point interpolants (Sec. 4.1), and
 *   - a history part carried by N_F = 2K + 1 Fourier modes alpha_k (eq. historySol1), advanced by
 *     an exact rotation plus a W-tap driving term (eqs. alphakEvolutionFormulas, hkcompdisc).
 * One step is a type-1 NUFFT (springs -> modes, eq. densco), the mode update, a type-2 NUFFT
 * (modes -> springs and receivers), the local sum and a sparse implicit density solve
 * (eq. linearSystem).  Free space adds the radiation projection of Sec. 4.4 every few steps.
 *
 * Conventions for every call:
 *   - Arrays are FP64, in the caller's spring order, contiguous.  A pointer documented as
 *     "device" must be a CUDA device (or managed) pointer usable from the current device; "host"
 *     pointers are ordinary (preferably pinned) host memory.
 *   - The plan copies every input it is given; the caller keeps ownership of its buffers and of
 *     every output buffer.  The plan owns its device memory and frees it in wave1d_destroy.
 *   - Work is queued on the plan's stream (wave1d_opts.stream; NULL is the legacy default
 *     stream).  Calls that return data to the host synchronise that stream.
 *   - Every call returns a wave1d_status.  Device-side faults of the numerics (non-finite
 *     densities) are latched in a device status word and reported by the next synchronising call
 *     (wave1d_sync, wave1d_read_receivers, wave1d_get_sigma, wave1d_solve).
 *   - Plans are not thread-safe; use one plan per host thread.
 */
#ifndef WAVE1D_H
#define WAVE1D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wave1d_plan_s* wave1d_plan_t;

/* boundary conditions: the periodic box [-pi, pi] (Sec. 2) or free space (Sec. 4.4) */
enum wave1d_bc { WAVE1D_PERIODIC = 0, WAVE1D_FREE = 1 };

enum wave1d_status {
    WAVE1D_OK = 0,
    WAVE1D_EINVAL = -1,        /* bad argument (NULL pointer, M < 1, dt <= 0, odd p, ...)       */
    WAVE1D_EDOMAIN = -2,       /* delta >= pi, or a free-space spring/receiver outside Omega   */
    WAVE1D_ENOMEM = -3,        /* device or host allocation failed / over the memory budget    */
    WAVE1D_ECUDA = -4,         /* a CUDA runtime call failed                                   */
    WAVE1D_ENOTCONV = -5,      /* the Jacobi sweeps of the implicit solve (local_weights = 1) did
                                  not converge within their limit (latched on the device)        */
    WAVE1D_ENONFINITE = -6,    /* a density became NaN or Inf (latched on the device)          */
    WAVE1D_EDONE = -7,         /* stepping past the Nt given to wave1d_plan                    */
    WAVE1D_EUNSUPPORTED = -9,  /* a size this build does not handle (see wave1d_strerror)      */
    WAVE1D_ETIMEOUT = -10      /* a bounded wait between the blocks of the one-launch step kernel
                                  ran out (latched on the device); the plan cannot continue      */
};

/* Optional parameters.  wave1d_opts_default fills the paper's defaults. */
typedef struct {
    int p;              /* local interpolation order, even, 2..16; default 8 (Sec. 6.3)            */
    double gamma;       /* fraction of K lost to windowing (Remark r:gamma); default 0.5           */
    int W;              /* window width in steps; 0 = ceil(2 ln(1/tol) / (pi gamma)) (eq. W)      */
    int NL;             /* Gauss-Legendre nodes of the local rule; 0 = W (Sec. 4.3)               */
    int Ng;             /* Gauss-Legendre nodes for p_k, q_k (eq. pkqkcomp); default 32           */
    int nufft_w;        /* spreading kernel width in fine-grid points; 0 = ceil(log10(1/tol)) + 1 */
    int rbc_period;     /* steps between radiation projections (Sec. 4.4); 0 = ceil(1.5 W)        */
    int max_block;      /* largest block of springs closer than dt solved directly; default 4096  */
    int64_t max_local_bytes; /* budget for stored local weights; default 16 GiB                  */
    int step_kernel;    /* 1 (default): ordinary steps run as one cooperative launch (history,
                           local sum and solve in one kernel); 0: one launch per stage           */
    void* stream;       /* cudaStream_t for all work of the plan; NULL = legacy default stream   */
    int precision;      /* 0 (default): FP64 throughout.  1: mixed, the history part's spreading
                           and interpolation in FP32 (the FP32 NUFFT kernels, width 7, about 1e-7
                           of the field; nufft_w must be 0 or 7), the FFTs, mode recurrence,
                           local sum and density solve as in FP64; steps run as per-stage
                           launches                                                              */
    int local_weights;  /* 0 (default): the local weights Q_m stored per pair and streamed every
                           step, the implicit blocks of I + S inverted at plan time.
                           1: no per-pair data.  The sources within delta of a spring are an index
                           window of the sorted springs; Q_m(d) comes from degree-7 polynomials in
                           d between the breakpoints of the rule (Sec. 4.1; within 1e-12 of
                           max |Q|), folded with each source's densities once per interval and
                           evaluated per pair in compensated FP32 pairs (local sums within about
                           2e-11 of the FP64 rule).  The implicit part is solved by Jacobi sweeps
                           until the largest change is below 1e-14 of the largest density
                           (WAVE1D_ENOTCONV after 40).  For layouts whose weights or blocks do
                           not fit (a million clustered springs: 1.3e10 pairs); steps run as
                           per-stage launches; wave1d_adjoint needs every stiffness > 0.
                           Batched plans also take 2: each instance's form chosen from its layout
                           (see wave1d_batch_plan)                                             */
    int spin_limit;     /* polls of a counter before a wait between the blocks of the one-launch
                           step kernel gives up and latches WAVE1D_ETIMEOUT; 0 = 2^22 (seconds)  */
    int hold_unit;      /* fault injection for tests, 0 = off: 1 makes the step kernel's column
                           pass leave its first unit uncounted, so the next phase's wait runs
                           out (WAVE1D_ETIMEOUT from the next synchronising call; the plan cannot
                           continue, the CUDA context stays usable)                            */
} wave1d_opts;

/* Derived sizes of a plan (read-only report). */
typedef struct {
    int64_t M, R, Nt, n;      /* springs, receivers, steps planned, steps taken                     */
    int K, NF, W, m_max, p, NL, Ng, nufft_w, nf, rbc_period;
    double dt, tol, b, delta;
    int64_t local_pairs;      /* (target, source) pairs within delta, springs only                   */
    int64_t local_weights;    /* stored local weights Q_m                                            */
    int64_t nearby_pairs;     /* pairs closer than dt (entries of S, eq. linearSystem)               */
    int64_t blocks, max_block;/* connected blocks of the nearby graph and the largest block size     */
    int64_t device_bytes;     /* device memory owned by the plan                                     */
    int64_t local_bytes;      /* bytes the local-sum kernel streams per step: weights, source lists,
                                 per-m counts, row offsets and its output                         */
    int64_t local_terms;      /* multiply-adds Q_m(d_jl) sigma_l^{n+1-m} of the local sum per step
                                 (pairs closer than delta times their non-zero m >= 1)            */
    int64_t solve_sweeps;     /* local_weights = 1: Jacobi sweeps of the last step's implicit solve
                                 (read from the device; waits for the plan's queued work), else 0 */
} wave1d_info;

/* Fill *o with defaults.  Returns WAVE1D_EINVAL if o is NULL. */
int wave1d_opts_default(wave1d_opts* o);

/*
 * Build a plan (Sec. 3-4): parameters b = ln(1/tol) (eq. b), K = floor(pi/dt) (eq. Kdt),
 * N_F = 2K + 1, W, delta = W dt (eq. W), the window tables, p_k and q_k (eq. pkqkcomp), the local
 * weights Q_m of every pair closer than delta (Sec. 4.1), the blocks of the implicit matrix
 * I + S (eq. linearSystem) and the NUFFT tables.  The densities start at zero (sigma(t <= 0) = 0).
 *   x, beta : host, M values each; positions (wrapped into [-pi, pi) for WAVE1D_PERIODIC) and
 *             stiffnesses (>= 0).  Free space needs |x_j| <= pi - 3 max(delta, W pi/K).
 *   bc      : WAVE1D_PERIODIC or WAVE1D_FREE.
 *   dt      : time step (> 0);  Nt: number of steps the plan may take (>= 1).
 *   tol     : window tolerance epsilon in (0, 0.1) (eq. b).
 *   opts    : NULL for defaults.
 *   out     : receives the plan handle (NULL on failure).
 */
int wave1d_plan(const double* x, const double* beta, int64_t M, int bc, double dt, int64_t Nt,
                double tol, const wave1d_opts* opts, wave1d_plan_t* out);

/*
 * Incident wave f(s) = sum_i amp_i exp(-(s - center_i)^2 / (2 width_i^2)), periodised over 2 pi
 * in the periodic box; it drives g_j(t) = beta_j f(x_j - t) (eq. gj, smooth f).  Host arrays of
 * n >= 0 values; n = 0 removes the incident wave.  Call before stepping.
 */
int wave1d_set_incident_gaussians(wave1d_plan_t plan, int n, const double* amp,
                                  const double* center, const double* width);

/*
 * Extra evaluation points for u = u_L + u_H (Sec. 3.1, last paragraph; eq. localSol2).
 * xr: host, R values (free space: inside Omega like the springs).  Call before stepping.
 */
int wave1d_set_receivers(wave1d_plan_t plan, const double* xr, int64_t R);

/*
 * Advance one step n -> n+1 (eq. linearSystem).  g_next: M values of g_j(t_{n+1}) in caller
 * order (host if g_on_device == 0, device otherwise), or NULL to use the incident wave.
 * Returns WAVE1D_EDONE once Nt steps have been taken.  Asynchronous.
 */
int wave1d_step(wave1d_plan_t plan, const double* g_next, int g_on_device);

/*
 * Advance nsteps steps driven by the incident wave, recording u at the receivers after each
 * step into u_rec[s * R + r] and, if sigma is not NULL, the densities into sigma[s * M + j]
 * (caller order).  Outputs are device pointers if out_on_device, host pointers otherwise.
 * Steps are replayed from captured CUDA graphs.  Synchronises the stream before returning.
 */
int wave1d_solve(wave1d_plan_t plan, int64_t nsteps, double* u_rec, double* sigma,
                 int out_on_device);

/* u at the receivers at the current time t_n (R values; device or host pointer).  Synchronises. */
int wave1d_read_receivers(wave1d_plan_t plan, double* u, int on_device);

/* sigma^n in caller order (M values; device or host pointer).  Synchronises. */
int wave1d_get_sigma(wave1d_plan_t plan, double* out, int on_device);

/* Wait for the plan's queued work and report a latched device status. */
int wave1d_sync(wave1d_plan_t plan);

/* Fill *info with the plan's derived sizes. */
int wave1d_get_info(wave1d_plan_t plan, wave1d_info* info);

/*
 * Copy an internal array to host memory for verification (synchronises).  Arrays in the plan's
 * internal (position-sorted) spring order unless stated; `count` is the number of doubles the
 * caller's buffer holds and must equal the size given here:
 *   WAVE1D_ARR_ALPHA      alpha_k^n, k = 0..K, interleaved (re, im)          2 (K+1)
 *   WAVE1D_ARR_ALPHA_P    alpha'_k^n                                          2 (K+1)
 *   WAVE1D_ARR_S_LAST     S_k^{n-1} of the last step, k = 0..K, (re, im)     2 (K+1)
 *   WAVE1D_ARR_UH         u_H(x_j, t_n) at springs, caller order              M
 *   WAVE1D_ARR_LOCAL      local explicit sum c_j of the last step, caller order M
 *   WAVE1D_ARR_SIGMA_RING sigma^{n-m}, m = 0..m_max, caller order, row m       (m_max+1) M
 *   WAVE1D_ARR_PERM       caller index of each sorted spring (as doubles)      M
 */
enum wave1d_array {
    WAVE1D_ARR_ALPHA = 0, WAVE1D_ARR_ALPHA_P = 1, WAVE1D_ARR_S_LAST = 2, WAVE1D_ARR_UH = 3,
    WAVE1D_ARR_LOCAL = 4, WAVE1D_ARR_SIGMA_RING = 5, WAVE1D_ARR_PERM = 6
};
int wave1d_inspect(wave1d_plan_t plan, int array, double* host_out, int64_t count);

/*
 * Per-stage device timing.  While enabled, steps run without graphs and CUDA events recorded on
 * the plan's stream between the stages of every step accumulate each stage's device time
 * (wave1d_stage order below).  wave1d_profile(plan, 1) resets the totals; (plan, 0) stops.
 * wave1d_profile_read copies the per-stage total milliseconds into ms[0..nstage-1] and the number
 * of profiled steps into *steps (synchronises).  nstage must be WAVE1D_NSTAGE.
 */
enum wave1d_stage {
    WAVE1D_STAGE_LOCAL = 0,      /* local explicit sum (Sec. 4.1)                     */
    WAVE1D_STAGE_SPREAD = 1,     /* type-1 spreading and the forward FFT's first pass */
    WAVE1D_STAGE_FFT_FWD = 2,    /* (merged into the neighbouring stages: zero)       */
    WAVE1D_STAGE_MODES = 3,      /* forward FFT rows, S_k, driving terms, rotation
                                    (Sec. 3), inverse FFT rows                        */
    WAVE1D_STAGE_RBC = 4,        /* radiation projection (Sec. 4.4), projection steps */
    WAVE1D_STAGE_FFT_INV = 5,    /* inverse FFT's last pass                           */
    WAVE1D_STAGE_INTERP = 6,     /* type-2 interpolation                              */
    WAVE1D_STAGE_SOLVE = 7,      /* forcing, right-hand side, block solve             */
    WAVE1D_STAGE_RECEIVERS = 8,  /* receiver readout                                  */
    WAVE1D_NSTAGE = 9
};
int wave1d_profile(wave1d_plan_t plan, int enable);
int wave1d_profile_read(wave1d_plan_t plan, double* ms, int nstage, int64_t* steps);

/*
 * Checkpoint and resume (no equation of the paper: the march's state between two steps).  The
 * state is what evolves with the march: the step counter, the latched status word, the density
 * rings (the last m_max + 1 steps of sigma, which the local part and the history part read), the
 * Fourier coefficients alpha, alpha' with the last W steps of S_k (eq. hkcompdisc), and the
 * receiver history of the current chunk.  Everything else is fixed by the plan's inputs.
 *   wave1d_state_size: *bytes = size of a state buffer for this plan.
 *   wave1d_state_save: buf: host memory of at least that size, written after the plan's queued
 *                      work has finished (synchronises the plan's stream).
 *   wave1d_state_load: buf: a buffer written by wave1d_state_save from a plan built with the same
 *                      inputs (positions, stiffnesses, bc, dt, tol, options, receivers); the plan
 *                      continues from the saved step.  WAVE1D_EINVAL if the buffer is too small,
 *                      not a state buffer, from a plan of other sizes, or past this plan's Nt.
 * The caller owns buf.  A resumed march reproduces the uninterrupted one bit for bit.
 */
int wave1d_state_size(wave1d_plan_t plan, size_t* bytes);
int wave1d_state_save(wave1d_plan_t plan, void* buf, size_t bytes);
int wave1d_state_load(wave1d_plan_t plan, const void* buf, size_t bytes);

/*
 * Reverse-time (adjoint) march of the discrete scheme: the gradients of a scalar loss L of the
 * receiver fields with respect to the stiffnesses and to the forcing, for a march of nsteps
 * steps from n = 0.  Each piece of a step is transposed in the real inner product and the steps
 * are taken in reverse order: the receiver readout (eq. localSol2), the implicit solve (eq.
 * linearSystem, transposed block inverses), the local sum (Sec. 4.1, transposed), the type-2 and
 * type-1 NUFFTs swapped (eqs. historySol1, densco), the projection of Sec. 4.4 and the mode
 * update (eqs. alphakEvolutionFormulas, hkcompdisc) transposed.  With rhsbar the adjoint of a
 * step's right-hand side, dL/dg^{n+1} = -rhsbar^n, and the stiffness, which enters a step through
 * rhs and S = diag(beta/2) Q_0, gives
 *   grad_beta_j = sum_n rhsbar_j^n sigma_j^{n+1} / beta_j                 (incident wave, eq. gj)
 *   grad_beta_j = sum_n rhsbar_j^n (sigma_j^{n+1} + g_j^{n+1}) / beta_j   (forcing vectors g)
 *   nsteps    : steps of the forward march, 1 <= nsteps <= Nt of the plan.
 *   sigma     : device, nsteps x M, row s = sigma^{s+1} in caller order (as wave1d_solve records it).
 *   g         : device, nsteps x M, row s = the forcing vector of step s + 1 given to wave1d_step
 *               (caller order), or NULL for a march driven by the incident wave.
 *   ubar      : device, nsteps x R, row s = dL/du_r(t_{s+1}) (NULL allowed when R = 0).
 *   grad_beta : device, M values, dL/dbeta_j in caller order (overwritten), or NULL.
 *   grad_g    : device, nsteps x M, row s = dL/dg^{s+1} in caller order (overwritten), or NULL.
 * At least one of grad_beta, grad_g.  grad_beta needs every stiffness > 0 (WAVE1D_EINVAL
 * otherwise); so does a plan without pair lists (opts.local_weights = 1), whose reverse march
 * transposes its range tables' local sum and its iterative implicit solve (the latter as the
 * forward sweeps on beta-scaled data; WAVE1D_ENOTCONV if they do not converge).  The plan's
 * tables are read and its march state is left alone.  Work arrays (a
 * ring of m_max + 1 density adjoints, the adjoint S ring and modes, an FP64 NUFFT plan of the
 * springs) are allocated for the call and freed before it returns.  No launch uses atomics: the
 * results are the same bit for bit from call to call.  Synchronises the plan's stream.
 */
int wave1d_adjoint(wave1d_plan_t plan, int64_t nsteps, const double* sigma, const double* g,
                   const double* ubar, double* grad_beta, double* grad_g);

/*
 * The reverse march without the stored densities: the forward march keeps its state every
 * `interval` steps (checkpoints), and the reverse pass marches each segment again from its
 * checkpoint, recording that segment's densities, before taking the segment's transposed steps.
 * Memory: ceil(nsteps / interval) checkpoints of the march state (the FP64 density ring of m_max + 1
 * rows, the S ring and the modes: about (m_max + 1) M + 2 (W + 2)(K + 1) doubles each) plus one
 * segment of interval x M densities, against nsteps x M for wave1d_adjoint; time: one more forward
 * march.  interval ~ sqrt(nsteps (m_max + 1)) balances the two terms.  Marches driven by the
 * incident wave (wave1d_solve); a march driven by forcing vectors takes wave1d_adjoint.
 *   wave1d_checkpoint_size:    *bytes = size of the device buffer of the checkpoints.
 *   wave1d_solve_checkpointed: from step 0 (a fresh plan, or one reloaded with a step-0 state),
 *       nsteps steps as wave1d_solve with sigma = NULL, recording u into u_rec (nsteps x R, device
 *       if u_on_device, else host; NULL allowed) and the checkpoints into ckpt (device, bytes >=
 *       wave1d_checkpoint_size).  Synchronises.
 *   wave1d_adjoint_checkpointed: the plan at the step its checkpointed march ended on, ckpt as
 *       written by that march (same nsteps and interval, WAVE1D_EINVAL otherwise): dL/dbeta and
 *       dL/dg as wave1d_adjoint with g = NULL (ubar, grad_beta, grad_g the same arrays).  The
 *       recomputed densities are those of the first march bit for bit, so the gradients equal
 *       wave1d_adjoint's from the stored densities bit for bit.  The plan's march state is put
 *       back to the end of the march before the call returns.  Work arrays (those of
 *       wave1d_adjoint, one segment of densities and a copy of the march state) are allocated for
 *       the call.  Synchronises.
 * The caller owns ckpt.
 */
int wave1d_checkpoint_size(wave1d_plan_t plan, int64_t nsteps, int64_t interval, size_t* bytes);
int wave1d_solve_checkpointed(wave1d_plan_t plan, int64_t nsteps, int64_t interval, double* u_rec,
                              int u_on_device, void* ckpt, size_t bytes);
int wave1d_adjoint_checkpointed(wave1d_plan_t plan, int64_t nsteps, int64_t interval, const void* ckpt,
                                size_t bytes, const double* ubar, double* grad_beta, double* grad_g);

/*
 * Standalone NUFFTs of the history part (Sec. 3.1) on fixed points, with the time-step plan's
 * Kaiser-Bessel kernel (eq. KB), fine grid and deconvolution:
 *   type-1 (eq. densco):       S_k = (1/2 pi) sum_j c_j e^{+i k x_j},  k = 0..K
 *   type-2 (eq. historySol1):  u_j = sum_{|k| <= K} alpha_k e^{-i k x_j},  alpha_{-k} = conj(alpha_k)
 * and their spreading (A1: grid G from c) and interpolation (A6: u from a grid) passes alone.
 *   wave1d_nufft_plan: x host, M positions (wrapped into [-pi, pi)); tol sets the kernel width as
 *       in wave1d_plan; precision 0 = FP64 (kernel weights precomputed), 1 = mixed (kernel values
 *       from FP32 Chebyshev series fitted to about 2e-7 of the kernel's peak, FP32 sums with the
 *       dominant terms compensated, FP64 FFT and deconvolution; tol >= 1e-6, else
 *       WAVE1D_EINVAL).  stream: cudaStream_t of every call (NULL = legacy default stream).
 *       Allocates the plan's device arrays.
 *   Point arrays (c, u) are device arrays of M FP64 in the plan's point order: point i is the
 *   caller's point perm[i] (wave1d_nufft_perm, host array of M).  S and alpha: device, K + 1
 *   complex (re, im interleaved).  grid: device, nf reals (wave1d_nufft_info).  Calls are queued on
 *   the plan's stream and do not synchronise; the plan owns its work arrays, so calls on one plan
 *   must not overlap.
 * Returns WAVE1D_EINVAL for bad arguments, WAVE1D_ENOMEM / WAVE1D_ECUDA on CUDA failures
 * (message: wave1d_nufft_strerror).
 */
typedef struct wave1d_nufft_s* wave1d_nufft_t;
int wave1d_nufft_plan(const double* x, int64_t M, int K, double tol, int precision, void* stream,
                      wave1d_nufft_t* out);
/*
 * Batched form: n_instances independent point sets with the same K and tol, one launch per pass
 * over all of them (the batched workload's instances, Sec. 6 shapes).  x: host, the instances'
 * positions one after another, instance i being x[offsets[i] .. offsets[i+1]) (offsets: host,
 * n_instances + 1 values, offsets[0] = 0, every instance with at least one point).  Point arrays
 * (c, u) hold all instances' points in the plan's order (perm keeps each instance within its
 * own segment); grid: n_instances x nf reals, instance-major; S and alpha: n_instances x (K + 1)
 * complex.  wave1d_nufft_plan(x, M, ...) is the one-instance case.
 */
int wave1d_nufft_plan_many(const double* x, const int64_t* offsets, int n_instances, int K, double tol,
                           int precision, void* stream, wave1d_nufft_t* out);
int wave1d_nufft_info(wave1d_nufft_t plan, int* nf, int* w, int* degree, double* kernel_err);
int wave1d_nufft_perm(wave1d_nufft_t plan, int64_t* perm);
int wave1d_nufft_spread(wave1d_nufft_t plan, const double* c, double* grid);
int wave1d_nufft_interp(wave1d_nufft_t plan, const double* grid, double* u);
int wave1d_nufft_type1(wave1d_nufft_t plan, const double* c, double* S);
int wave1d_nufft_type2(wave1d_nufft_t plan, const double* alpha, double* u);
int wave1d_nufft_destroy(wave1d_nufft_t plan);
const char* wave1d_nufft_strerror(void);
/*
 * Autotuner of the spreading's work split: the cells and the points a cell range is cut at (the
 * spreading's tile width and bin size).  Each of nine candidate pairs, at or below the kernels'
 * shared-memory capacities (mixed: 60/120/240 cells x 512/1024/2048 points; FP64: 32/64/128 x
 * 1024/2048/4096), re-cuts the plan's ranges.  Each is timed over `reps` spreads of c (device,
 * plan's point order) into grid (device, overwritten), after one untimed spread, with CUDA events
 * on the plan's stream.  The fastest stays in the plan; *cells and *points (may be NULL) receive
 * its caps.  Results change only in rounding: every candidate tiles the grids completely.
 * Synchronises the plan's stream.
 */
int wave1d_nufft_autotune(wave1d_nufft_t plan, const double* c, double* grid, int reps, int* cells,
                          int* points);

/*
 * Type-1 NUFFT of device arrays without any memory allocation (the paper has no counterpart; it
 * is a service for callers that cannot allocate device memory — code running under a memory
 * budget reserved up front, or in a loop that must not take the implicit device synchronisation
 * cudaMalloc/cudaFree can cause).
 *   S[2k], S[2k+1] = Re, Im of (1/2 pi) sum_j c[j] e^{i k x[j]},  k = 0..K
 * computed with the spreading kernel, fine grid and FFT a plan of the same K and tol uses.  The
 * spreading adds into the fine grid with FP64 atomics, so the order of those additions, and the
 * last bits of S (about 1e-16 of max |S|), can differ from call to call: unlike every other call
 * of this library, the result is not bitwise reproducible.
 *   x, c : device, M values (x read periodically on [-pi, pi)); S: device, 2 (K+1) values.
 *   stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 * All intermediates live in one file-scope device array of 2 MiB that every GPU loading the
 * library keeps until exit; fine grids above 65536 points (K > 16383) return
 * WAVE1D_EUNSUPPORTED.  The first call on a device looks up that array's address (with that
 * device current); make it before any stream capture.  The array is shared by all calls and keeps
 * the last call's contents, so calls that overlap on the GPU race; serialise them on one stream.
 * No cudaMalloc, cudaFree or other allocating routine is called.
 */
int wave1d_nufft1_noalloc(const double* x, const double* c, int64_t M, int K, double tol,
                          double* S, void* stream);

/*
 * Batched march: n_inst independent instances in the periodic box, each with its own springs,
 * stiffnesses, one incident Gaussian (eq. gj) and receivers, sharing dt, Nt, tol and the options,
 * advance together.  One step of all instances is one pass of launches: the local sum (Sec. 4.1)
 * and the block solve (eq. linearSystem) over the instances' joined tables, and each instance's
 * history part (Sec. 3) with the spreading and interpolation of all instances in one launch each
 * (the batched NUFFT plan above).  With opts.step_kernel = 1 (the default), where the device
 * launches cooperative grids and the kernel width is 7 .. 14 (tol 1e-6 .. 1e-13), the whole step
 * of every instance is one persistent cooperative launch instead (the same unit bodies in the same
 * order, so the same bits); its waits between blocks are bounded by opts.spin_limit and latch
 * WAVE1D_ETIMEOUT.  Either way the step is captured once in a CUDA graph and replayed.
 *   offsets : host, n_inst + 1 values, offsets[0] = 0; instance i holds springs
 *             [offsets[i], offsets[i+1]) of x and beta (host, positions wrapped into [-pi, pi)),
 *             at least one spring each.
 *   pulse   : host, n_inst x 3: amplitude, centre, width of instance i's incident Gaussian.
 *   r_offsets, xr : host receivers, instance i's being xr[r_offsets[i] .. r_offsets[i+1]) (at
 *             least one each), or r_offsets = NULL for none.
 *   dt, Nt, tol : as wave1d_plan.  opts: NULL or as wave1d_plan with precision 0 and nufft_w 0
 *                 (others: WAVE1D_EINVAL), and local_weights:
 *       0 (default): every instance in the joined tables above (stored weights);
 *       1: every instance is a plan of its own without pair lists (opts.local_weights = 1 of
 *          wave1d_plan), stepped as one branch of the step's graph, concurrently with the others;
 *       2: per instance, from its positions: without pair lists when its largest block of springs
 *          closer than dt has more than opts.max_block members, when more than 2^19 ordered pairs
 *          of its springs are closer than delta = W dt, or when its stored weights would pass
 *          what is left of opts.max_local_bytes; the joined tables otherwise.
 *       The joined instances' step runs first (the one persistent launch), then the branches.
 * Every instance's derived sizes (K, W, fine grid) are the same, since they depend on dt, tol and
 * p only.  The springs' and receivers' global order is instance-major in the caller's order.
 * Returns WAVE1D_EINVAL / EDOMAIN / ENOMEM / ECUDA like wave1d_plan (message: wave1d_batch_strerror).
 */
typedef struct wave1d_batch_s* wave1d_batch_t;
int wave1d_batch_plan(int n_inst, const int64_t* offsets, const double* x, const double* beta,
                      const double* pulse, const int64_t* r_offsets, const double* xr, double dt,
                      int64_t Nt, double tol, const wave1d_opts* opts, wave1d_batch_t* out);
/*
 * Advance nsteps steps; u_rec[s * R + r] (R: all receivers) and, if sigma is not NULL,
 * sigma[s * M + j] (M: all springs) after step s + 1, device or host pointers as out_on_device.
 * Synchronises; WAVE1D_EDONE past Nt, WAVE1D_ENONFINITE if a density became non-finite,
 * WAVE1D_ENOTCONV if an instance without pair lists did not converge, WAVE1D_ETIMEOUT if a wait of
 * the one-launch step ran out.
 */
int wave1d_batch_solve(wave1d_batch_t plan, int64_t nsteps, double* u_rec, double* sigma,
                       int out_on_device);
int wave1d_batch_destroy(wave1d_batch_t plan);
const char* wave1d_batch_strerror(void);
/* 1 if the joined instances' steps run as one persistent launch (see wave1d_batch_plan), 0 if as
 * one launch per pass or if no instance is joined, WAVE1D_EINVAL for a NULL plan. */
int wave1d_batch_step_kernel(wave1d_batch_t plan);
/* forms: host, n_inst values, 0 for an instance in the joined tables, 1 for one marched as its own
 * plan without pair lists (opts.local_weights of wave1d_batch_plan).  WAVE1D_EINVAL for NULL. */
int wave1d_batch_forms(wave1d_batch_t plan, int* forms);

/* Free the plan and its device memory (synchronises).  NULL is accepted. */
int wave1d_destroy(wave1d_plan_t plan);

/* Static description of a status code, or of the last error detail of the calling thread. */
const char* wave1d_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* WAVE1D_H */
