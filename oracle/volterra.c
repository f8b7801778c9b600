/*
 * Oracle A: direct all-to-all time march of the point-spring Volterra system.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain FP64 reference that the
 * tests, the smoke check and the CPU-baseline leg of the benchmark use to judge the
 * CUDA library.  The product path never links, loads or calls it, and it shares no
 * code with the CUDA sources.
 *
 * What it computes (Sec. 1, eq. IEfree; Sec. 2, eq. periodicIE):
 *
 *   -sigma_j(t) - (beta_j/2) sum_l sum_images int_0^{t - |x_j - x_l - 2 pi m|} sigma_l = g_j(t)
 *
 * with g_j(t) = beta_j f(x_j - t) (eq. gj; f is smooth so [d_x u_inc] = 0), f periodised
 * over 2 pi in the periodic box (Sec. 2).  Free space keeps the single image m = 0.
 *
 * Discretisation (Sec. 4.1 and Sec. 5): sigma is sampled at t_q = q dt, with sigma^q = 0 for
 * q <= 0 (the densities switch on smoothly, Sec. 2).  Each running integral
 * I_l(s) = int_0^s sigma_l is the exact integral of a piecewise polynomial interpolant: on the
 * interval [t_a, t_{a+1}] it is the degree p-1 Lagrange polynomial through the p nearest grid
 * samples, i.e. the indices a-p/2+1 .. a+p/2 for even p, moved down so that no index exceeds
 * the newest usable one.  The newest usable index is n+1 (the unknown) for "nearby" pairs at
 * distance < dt and n for all others, which is the same causal split as eq. periodicIE_disc.
 * For p = 1 the interpolant is the value at the left end of each interval (Sec. 5.1).
 * Exact integration uses a Gauss-Legendre rule exact for degree p-1 (nodes passed in).
 *
 * The sigma^{n+1} terms of nearby pairs give a small linear system, solved by Gaussian
 * elimination with partial pivoting on each connected block of nearby springs.
 *
 * Recurrence of the Remark in Sec. 1: the integrals over intervals whose centred stencil is
 * complete never change again, so they are kept in running prefix sums per spring.
 *
 * Receivers: u(x_r, t_{n+1}) = 1/2 sum_l sum_images I_l(t_{n+1} - |x_r - x_l - 2 pi m|)
 * (eq. singleLayerSol / SLPp), evaluated after sigma^{n+1} is known, with the same stencil rule.
 *
 * Complex-step build (compiled a second time with -DORACLE_COMPLEX_STEP): the stiffnesses,
 * densities, prefix sums, receiver fields and the block solve hold complex numbers, the geometry
 * and quadrature stay real, and the entry point is oracle_volterra_march_cs.  Every operation on
 * the complex values is a sum or a product, so with beta_j + i h the imaginary part of any output
 * divided by h is its derivative with respect to beta_j up to O(h^2), free of cancellation
 * (Squire and Trapp, SIAM Rev. 40, 1998).  Pivots are chosen by the real part, the same choice
 * as the real build.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_COMPLEX_STEP
#include <complex.h>
typedef double _Complex scalar_t;
#define PIVOT_MAG(v) fabs(creal(v))
#define MARCH_ENTRY oracle_volterra_march_cs
#else
typedef double scalar_t;
#define PIVOT_MAG(v) fabs(v)
#define MARCH_ENTRY oracle_volterra_march
#endif

#define TWO_PI 6.283185307179586476925286766559

/* incident profile f(s) = sum_p amp_p exp(-(s - c_p)^2 / (2 w_p^2)); 2 pi periodised if asked */
static double incident(double s, int np, const double* amp, const double* c, const double* w,
                       int periodic)
{
    double f = 0.0;
    for (int q = 0; q < np; q++) {
        if (!periodic) {
            double z = (s - c[q]) / w[q];
            f += amp[q] * exp(-0.5 * z * z);
        } else {
            double span = 40.0 * w[q];
            long m0 = (long)floor((c[q] - s - span) / TWO_PI);
            long m1 = (long)ceil((c[q] - s + span) / TWO_PI);
            for (long m = m0; m <= m1; m++) {
                double z = (s + TWO_PI * (double)m - c[q]) / w[q];
                f += amp[q] * exp(-0.5 * z * z);
            }
        }
    }
    return f;
}

/* first index of the p-point stencil of interval [t_a, t_{a+1}] given the newest usable index */
static long stencil_start(long a, int p, long newest)
{
    if (p == 1) return a;
    long q0 = a - p / 2 + 1;
    if (q0 + p - 1 > newest) q0 = newest - p + 1;
    return q0;
}

/* largest sample index the unshifted stencil of interval a touches */
static long stencil_top(long a, int p)
{
    return (p == 1) ? a : a + p / 2;
}

/*
 * integral over y in [a, a + theta] (time in units of dt) of the interpolant built on the
 * stencil for `newest`; sig[q] holds sigma^q for q >= 1, indices <= 0 read as zero.  The
 * coefficient multiplying the sample with index `imp` is returned in *cimp instead of being
 * multiplied by sig (pass imp = -1 to use sig for every index).  Result is in units of dt.
 */
static scalar_t interval_integral(const scalar_t* sig, long a, double theta, int p, long newest,
                                long imp, double* cimp, int ng, const double* gx, const double* gw)
{
    long q0 = stencil_start(a, p, newest);
    scalar_t acc = 0.0;
    for (int i = 0; i < ng; i++) {
        double y = (double)a + 0.5 * theta * (1.0 + gx[i]);
        double wt = 0.5 * theta * gw[i];
        for (int r = 0; r < p; r++) {
            long q = q0 + r;
            double L = 1.0;
            for (int s = 0; s < p; s++) {
                if (s == r) continue;
                L *= (y - (double)(q0 + s)) / (double)(r - s);
            }
            if (q == imp) {
                *cimp += wt * L;
            } else if (q >= 1) {
                acc += wt * L * sig[q];
            }
        }
    }
    return acc;
}

/* union-find for the blocks of springs coupled through sigma^{n+1} */
static long uf_find(long* parent, long i)
{
    while (parent[i] != i) {
        parent[i] = parent[parent[i]];
        i = parent[i];
    }
    return i;
}

/* dense Gaussian elimination with partial pivoting, A is n x n row-major, b overwritten */
static int dense_solve(int n, scalar_t* A, scalar_t* b)
{
    for (int k = 0; k < n; k++) {
        int piv = k;
        double best = PIVOT_MAG(A[k * n + k]);
        for (int i = k + 1; i < n; i++) {
            if (PIVOT_MAG(A[i * n + k]) > best) { best = PIVOT_MAG(A[i * n + k]); piv = i; }
        }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < n; c++) {
                scalar_t t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t;
            }
            scalar_t t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; i++) {
            scalar_t f = A[i * n + k] / A[k * n + k];
            if (f == 0.0) continue;
            for (int c = k; c < n; c++) A[i * n + c] -= f * A[k * n + c];
            b[i] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        scalar_t s = b[k];
        for (int c = k + 1; c < n; c++) s -= A[k * n + c] * b[c];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

/* list of (source, distance) pairs a target sees, all images within reach of t_end */
typedef struct { long l; double d; } pair_t;

static long collect_pairs(double xt, long M, const double* x, int periodic, double t_end,
                          pair_t* out)
{
    long cnt = 0;
    for (long l = 0; l < M; l++) {
        if (!periodic) {
            double d = fabs(xt - x[l]);
            if (d <= t_end) { out[cnt].l = l; out[cnt].d = d; cnt++; }
        } else {
            long mlim = (long)ceil((t_end + TWO_PI) / TWO_PI) + 1;
            for (long m = -mlim; m <= mlim; m++) {
                double d = fabs(xt - x[l] - TWO_PI * (double)m);
                if (d <= t_end) { out[cnt].l = l; out[cnt].d = d; cnt++; }
            }
        }
    }
    return cnt;
}

/*
 * Running integral I_l(s) at s = t_{n+1} - d, split into the part from known samples (returned,
 * units of dt) and the coefficient of sigma_l^{n+1} (*cimp, units of dt).
 * sig_l: samples of spring l (index q at sig_l[q]); P_l: prefix sums of final intervals;
 * afin: number of final intervals stored in P_l.
 */
static scalar_t running_integral(const scalar_t* sig_l, const scalar_t* P_l, long afin, long n,
                               double d, double dt, int p, int use_imp, double* cimp, int ng,
                               const double* gx, const double* gw)
{
    double y = (double)(n + 1) - d / dt;
    if (y <= 0.0) return 0.0;
    long as = (long)floor(y);
    double theta = y - (double)as;
    long newest = (d < dt) ? n + 1 : n;
    long imp = use_imp ? n + 1 : -1;
    long a0 = as < afin ? as : afin;
    scalar_t acc = P_l[a0];
    for (long a = a0; a < as; a++)
        acc += interval_integral(sig_l, a, 1.0, p, newest, imp, cimp, ng, gx, gw);
    if (theta > 0.0)
        acc += interval_integral(sig_l, as, theta, p, newest, imp, cimp, ng, gx, gw);
    return acc;
}

/*
 * March Nt steps.  Outputs sigma_out[n * M + j] for n = 0..Nt and u_out[n * R + r].
 * g_in (optional, (Nt+1) x M) replaces the incident forcing (used for manufactured solutions).
 * gx, gw: Gauss-Legendre nodes/weights on [-1, 1] with ng >= p/2 + 1.
 * Returns 0, or -1 on a singular block, -2 on bad arguments, -3 on allocation failure.
 */
int MARCH_ENTRY(long M, const double* x, const scalar_t* beta, int periodic, double dt,
                          long Nt, int p, int npulse, const double* amp, const double* center,
                          const double* width, const double* g_in, long R, const double* xr,
                          int ng, const double* gx, const double* gw, scalar_t* sigma_out,
                          scalar_t* u_out)
{
    if (M < 1 || Nt < 0 || dt <= 0.0 || p < 1 || (p > 1 && (p % 2) != 0)) return -2;
    long stride = Nt + 2;                       /* sig[l * stride + q], q = 0..Nt+1 */
    long pstride = Nt + 3;                      /* P[l * pstride + a],  a = 0..Nt+2 */
    double T = (double)Nt * dt;
    long per_src = periodic ? (long)floor(T / (0.5 * TWO_PI)) + 3 : 1;
    scalar_t* sig = (scalar_t*)calloc((size_t)M * stride, sizeof(scalar_t));
    scalar_t* P = (scalar_t*)calloc((size_t)M * pstride, sizeof(scalar_t));
    scalar_t* rhs = (scalar_t*)malloc(sizeof(scalar_t) * (size_t)M);
    /* nearby pairs (distance < dt over the nearest image), CSR by target; geometry only */
    long* nb_ptr = (long*)calloc((size_t)M + 1, sizeof(long));
    if (!sig || !P || !rhs || !nb_ptr) return -3;
    for (long j = 0; j < M; j++)
        for (long l = 0; l < M; l++) {
            double d = fabs(x[j] - x[l]);
            if (periodic) { d = fmod(d, TWO_PI); if (TWO_PI - d < d) d = TWO_PI - d; }
            if (d < dt) nb_ptr[j + 1]++;
        }
    for (long j = 0; j < M; j++) nb_ptr[j + 1] += nb_ptr[j];
    long nnb = nb_ptr[M];
    long* nb_l = (long*)malloc(sizeof(long) * (size_t)(nnb + 1));
    double* nb_d = (double*)malloc(sizeof(double) * (size_t)(nnb + 1));
    scalar_t* nb_c = (scalar_t*)malloc(sizeof(scalar_t) * (size_t)(nnb + 1));
    if (!nb_l || !nb_d || !nb_c) return -3;
    for (long j = 0; j < M; j++) {
        long e = nb_ptr[j];
        for (long l = 0; l < M; l++) {
            double d = fabs(x[j] - x[l]);
            if (periodic) { d = fmod(d, TWO_PI); if (TWO_PI - d < d) d = TWO_PI - d; }
            if (d < dt) { nb_l[e] = l; nb_d[e] = d; e++; }
        }
    }
    /* blocks of springs coupled through sigma^{n+1}: union-find, then members by block */
    long* parent = (long*)malloc(sizeof(long) * (size_t)M);
    long* bstart = (long*)calloc((size_t)M + 1, sizeof(long));
    long* members = (long*)malloc(sizeof(long) * (size_t)M);
    long* local = (long*)malloc(sizeof(long) * (size_t)M);
    long* fill = (long*)malloc(sizeof(long) * (size_t)M);
    if (!parent || !bstart || !members || !local || !fill) return -3;
    for (long j = 0; j < M; j++) parent[j] = j;
    for (long j = 0; j < M; j++)
        for (long e = nb_ptr[j]; e < nb_ptr[j + 1]; e++) {
            long a = uf_find(parent, j), b = uf_find(parent, nb_l[e]);
            if (a != b) parent[a] = b;
        }
    for (long j = 0; j < M; j++) bstart[uf_find(parent, j) + 1]++;
    for (long j = 0; j < M; j++) bstart[j + 1] += bstart[j];
    for (long j = 0; j < M; j++) fill[j] = bstart[j];
    for (long j = 0; j < M; j++) {
        long rt = uf_find(parent, j);
        local[j] = fill[rt] - bstart[rt];
        members[fill[rt]++] = j;
    }

    int status = 0;
    long afin = 0;
    for (long j = 0; j < M; j++) sigma_out[j] = 0.0;
    for (long r = 0; r < R; r++) u_out[r] = 0.0;

    for (long n = 0; n < Nt; n++) {
        double t1 = (double)(n + 1) * dt;
        /* explicit parts (every pair except the nearby image) and nearby coefficients */
        #pragma omp parallel
        {
            pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)M * per_src + 16);
            #pragma omp for schedule(dynamic, 4)
            for (long j = 0; j < M; j++) {
                long np_ = collect_pairs(x[j], M, x, periodic, t1, pairs);
                scalar_t known = 0.0;
                for (long e = 0; e < np_; e++) {
                    if (pairs[e].d < dt) continue;          /* nearby images handled below */
                    double cimp = 0.0;
                    known += running_integral(sig + pairs[e].l * stride, P + pairs[e].l * pstride,
                                              afin, n, pairs[e].d, dt, p, 1, &cimp, ng, gx, gw);
                }
                for (long e = nb_ptr[j]; e < nb_ptr[j + 1]; e++) {
                    double cimp = 0.0;
                    known += running_integral(sig + nb_l[e] * stride, P + nb_l[e] * pstride, afin,
                                              n, nb_d[e], dt, p, 1, &cimp, ng, gx, gw);
                    nb_c[e] = 0.5 * beta[j] * dt * cimp;
                }
                scalar_t g = g_in ? g_in[(n + 1) * M + j]
                                : beta[j] * incident(x[j] - t1, npulse, amp, center, width, periodic);
                rhs[j] = -g - 0.5 * beta[j] * dt * known;
            }
            free(pairs);
        }
        /* (I + S) sigma^{n+1} = rhs, block by block */
        #pragma omp parallel for schedule(dynamic, 1)
        for (long rt = 0; rt < M; rt++) {
            long b0 = bstart[rt], nbk = bstart[rt + 1] - b0;
            if (nbk == 0) continue;
            scalar_t* A = (scalar_t*)calloc((size_t)nbk * nbk, sizeof(scalar_t));
            scalar_t* bb = (scalar_t*)malloc(sizeof(scalar_t) * (size_t)nbk);
            for (long i = 0; i < nbk; i++) {
                long j = members[b0 + i];
                A[i * nbk + i] = 1.0;
                bb[i] = rhs[j];
                for (long e = nb_ptr[j]; e < nb_ptr[j + 1]; e++)
                    A[i * nbk + local[nb_l[e]]] += nb_c[e];
            }
            if (dense_solve((int)nbk, A, bb) != 0) status = -1;
            for (long i = 0; i < nbk; i++) sig[members[b0 + i] * stride + (n + 1)] = bb[i];
            free(A);
            free(bb);
        }
        for (long j = 0; j < M; j++) sigma_out[(n + 1) * M + j] = sig[j * stride + (n + 1)];

        /* receivers with sigma^{n+1} known */
        #pragma omp parallel
        {
            pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)M * per_src + 16);
            #pragma omp for
            for (long r = 0; r < R; r++) {
                long np_ = collect_pairs(xr[r], M, x, periodic, t1, pairs);
                scalar_t u = 0.0;
                for (long e = 0; e < np_; e++) {
                    double dummy = 0.0;
                    u += running_integral(sig + pairs[e].l * stride, P + pairs[e].l * pstride, afin,
                                          n, pairs[e].d, dt, p, 0, &dummy, ng, gx, gw);
                }
                u_out[(n + 1) * R + r] = 0.5 * dt * u;
            }
            free(pairs);
        }

        /* intervals whose centred stencil is now complete join the prefix sums */
        while (afin <= Nt && stencil_top(afin, p) <= n + 1) {
            #pragma omp parallel for
            for (long l = 0; l < M; l++) {
                double dummy = 0.0;
                scalar_t F = interval_integral(sig + l * stride, afin, 1.0, p, n + 1, -1, &dummy,
                                             ng, gx, gw);
                P[l * pstride + afin + 1] = P[l * pstride + afin] + F;
            }
            afin++;
        }
    }
    free(sig); free(P); free(rhs); free(nb_ptr); free(nb_l); free(nb_d); free(nb_c);
    free(parent); free(bstart); free(members); free(local); free(fill);
    return status;
}
