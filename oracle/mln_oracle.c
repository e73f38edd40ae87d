/*
 * MLN oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU solver of the one-dimensional Maxwell-Liouville-von
 * Neumann equations in full density-matrix form (N x N complex rho per cell),
 * written to be checked against the paper by eye. It is used by the test
 * suite, by the smoke check and by the CPU-baseline leg of the benchmark, and
 * never by the product path. It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (Riesch & Jirauschek, "Numerical Method for the
 * Maxwell-Liouville-von Neumann Equations using Efficient Matrix Exponential
 * Computations"):
 *   - Maxwell's curl equations in 1D (Sec. 2, Eq. 1) on the staggered FDTD grid
 *     of Fig. 1: E_z at integer cells and integer time levels, H_y between
 *     cells at half time levels, rho (and dP/dt) at the E_z cells, half a time
 *     step apart from E_z.
 *   - The Liouville-von Neumann equation (Sec. 2, Eq. 2) with
 *     H = H0 - mu E_z, advanced by the symmetric Strang splitting of Sec. 4.1
 *     (Eqs. 21-23): half a step of the field-free part L0 + G, a full step of
 *     the interaction part with the midpoint field E_z^n (Eq. 22), and half a
 *     step of L0 + G again. Here each sub-flow is applied to rho itself, not to
 *     the adjoint vector d: the field-free flow is the N^2 x N^2 superoperator
 *     exponential exp((L0 + G) dt/2), computed once; the interaction flow is
 *     rho -> V rho V^+ with V = exp(+i mu E_z^n dt / hbar), the exact solution
 *     of d rho/dt = -(i/hbar)[-mu E_z, rho] for a constant field. Every matrix
 *     exponential is a generic scaling-and-squaring diagonal Pade(13)
 *     approximant (the paper's "pade" baseline idea, Sec. 4.1 and Sec. 5), so
 *     no structure of U or of the adjoint representation is used.
 *   - The polarisation source dP/dt = N_a Tr{mu (L0(rho) + G(rho))}
 *     (Sec. 2, Eqs. 3-5), evaluated on rho^{n+1/2}.
 *
 * Readings of points the paper leaves open (the paper is silent on each):
 *   - order in a step: H^{n+1/2} from E^n; rho^{n-1/2} -> rho^{n+1/2} with E^n;
 *     dP/dt^{n+1/2} from rho^{n+1/2}; E^{n+1} from H^{n+1/2} and dP/dt^{n+1/2};
 *   - conductivity is averaged semi-implicitly:
 *     E^{n+1}(1 + s) = E^n(1 - s) + dt/eps (dH/dx - dP/dt), s = sigma dt/(2 eps);
 *   - boundaries: periodic ring; or "open": E at cell 0 is driven only by a
 *     hard source (held otherwise) and the right end uses the first-order Mur
 *     condition; or "window": both end cells held, used to compute a single
 *     interior cell of a larger grid from its light cone;
 *   - source sample n is applied after the E update that produces E^{n+1}
 *     (hard: replace, soft: add);
 *   - vacuum cells (outside [medium_begin, medium_end)) carry no rho and
 *     contribute dP/dt = 0.
 *
 * Field solver: besides the FDTD differences of Fig. 1, the pseudo-spectral
 * (PSTD) variant that Secs. 1 and 3 say the method carries over to: on a
 * periodic grid of n cells, dE/dx at the H points and dH/dx at the E points are
 * the derivatives of the trigonometric interpolants of the samples, i.e. the
 * DFT multiplied by i k e^{+i k dx/2} (E -> H points) or i k e^{-i k dx/2}
 * (H -> E points), k = 2 pi m / (n dx) for m = 0 .. n/2 and 2 pi (m - n) /
 * (n dx) above; the time stepping and the Liouville step are unchanged. Here
 * each derivative is a circulant matrix whose first column comes from that
 * definition (inverse DFT of the multipliers, summed term by term), applied
 * by a plain O(n^2) sum: no FFT.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_HBAR 1.054571817e-34
#define ORC_EPS0 8.8541878128e-12
#define ORC_MU0 1.25663706212e-6

enum { ORC_BC_PERIODIC = 0, ORC_BC_OPEN = 1, ORC_BC_WINDOW = 2 };
enum { ORC_SRC_NONE = 0, ORC_SRC_HARD = 1, ORC_SRC_SOFT = 2 };
enum { ORC_FDTD = 0, ORC_PSTD = 1 };

typedef struct {
    int N;
    const double *H0;  /* N*N complex (re, im interleaved), row-major, J */
    const double *mu;  /* N*N complex, C m */
    const double *G;   /* N^2 x N^2 complex on row-major vec(rho), 1/s; NULL = none */
    double N_a;        /* m^-3 */
    long n_cells, medium_begin, medium_end;
    double dx, dt, eps_r, mu_r, sigma;
    int boundary, source_kind;
    long source_cell;
    int maxwell;       /* ORC_FDTD or ORC_PSTD (periodic grids only) */
} orc_problem;

/* ---------------------------------------------------------------- matrices */

static void mat_mul(int n, const cplx *A, const cplx *B, cplx *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx s = 0;
            for (int k = 0; k < n; ++k)
                s += A[i * n + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

static double norm1(int n, const cplx *A)
{
    double best = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < n; ++i)
            s += cabs(A[i * n + j]);
        if (s > best)
            best = s;
    }
    return best;
}

/* Solve Q X = P for X (n x n), Gaussian elimination with partial pivoting.
 * Q and P are overwritten. Returns 0 on success, -1 if Q is singular. */
static int solve(int n, cplx *Q, cplx *P, cplx *X)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(Q[r * n + c]) > cabs(Q[piv * n + c]))
                piv = r;
        if (cabs(Q[piv * n + c]) == 0.0)
            return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                cplx t = Q[c * n + k]; Q[c * n + k] = Q[piv * n + k]; Q[piv * n + k] = t;
                t = P[c * n + k]; P[c * n + k] = P[piv * n + k]; P[piv * n + k] = t;
            }
        }
        for (int r = c + 1; r < n; ++r) {
            cplx f = Q[r * n + c] / Q[c * n + c];
            for (int k = c; k < n; ++k)
                Q[r * n + k] -= f * Q[c * n + k];
            for (int k = 0; k < n; ++k)
                P[r * n + k] -= f * P[c * n + k];
        }
    }
    for (int r = n - 1; r >= 0; --r)
        for (int k = 0; k < n; ++k) {
            cplx s = P[r * n + k];
            for (int c = r + 1; c < n; ++c)
                s -= Q[r * n + c] * X[c * n + k];
            X[r * n + k] = s / Q[r * n + r];
        }
    return 0;
}

/*
 * exp(A) by scaling and squaring with the diagonal [13/13] Pade approximant
 * (Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179): A is scaled by 2^-s so
 * that its 1-norm is at most 1/2, r13(B) = q13(B)^-1 p13(B) with
 * p13(B) = sum_k c_k B^k, q13(B) = p13(-B),
 * c_k = (26-k)! 13! / (26! k! (13-k)!), then squared s times.
 * The powers are formed one by one, without Higham's blocking, so that the
 * steps are visible.
 */
static int expm_c(int n, const cplx *A, cplx *X)
{
    const int m = 13;
    double c[14];
    c[0] = 1.0;
    for (int k = 1; k <= m; ++k)
        c[k] = c[k - 1] * (double)(m - k + 1) / ((double)k * (double)(2 * m - k + 1));

    double nrm = norm1(n, A);
    int s = 0;
    while (ldexp(nrm, -s) > 0.5)
        ++s;

    size_t nn = (size_t)n * n;
    cplx *B = malloc(nn * sizeof(cplx));
    cplx *Bk = malloc(nn * sizeof(cplx));
    cplx *T = malloc(nn * sizeof(cplx));
    cplx *P = malloc(nn * sizeof(cplx));
    cplx *Q = malloc(nn * sizeof(cplx));
    if (!B || !Bk || !T || !P || !Q) {
        free(B); free(Bk); free(T); free(P); free(Q);
        return -2;
    }
    double scale = ldexp(1.0, -s);
    for (size_t i = 0; i < nn; ++i)
        B[i] = A[i] * scale;

    /* k = 0 term: identity */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            Bk[i * n + j] = (i == j) ? 1.0 : 0.0;
            P[i * n + j] = (i == j) ? c[0] : 0.0;
            Q[i * n + j] = (i == j) ? c[0] : 0.0;
        }
    for (int k = 1; k <= m; ++k) {
        mat_mul(n, Bk, B, T);
        memcpy(Bk, T, nn * sizeof(cplx));
        double sign = (k % 2) ? -1.0 : 1.0;
        for (size_t i = 0; i < nn; ++i) {
            P[i] += c[k] * Bk[i];
            Q[i] += sign * c[k] * Bk[i];
        }
    }
    int rc = solve(n, Q, P, X);
    for (int r = 0; r < s && rc == 0; ++r) {
        mat_mul(n, X, X, T);
        memcpy(X, T, nn * sizeof(cplx));
    }
    free(B); free(Bk); free(T); free(P); free(Q);
    return rc;
}

static void load_c(size_t n, const double *src, cplx *dst)
{
    for (size_t i = 0; i < n; ++i)
        dst[i] = src[2 * i] + I * src[2 * i + 1];
}

static void store_c(size_t n, const cplx *src, double *dst)
{
    for (size_t i = 0; i < n; ++i) {
        dst[2 * i] = creal(src[i]);
        dst[2 * i + 1] = cimag(src[i]);
    }
}

/* --------------------------------------------------------- superoperators */

/*
 * L0 + G as an N^2 x N^2 matrix acting on row-major vec(rho) (Sec. 2, Eq. 2):
 * (L0 rho)_{jk} = -(i/hbar) sum_l (H0_{jl} rho_{lk} - rho_{jl} H0_{lk}),
 * so the entry at row (j,k), column (l,m) is
 * -(i/hbar) (H0_{jl} delta_{km} - delta_{jl} H0_{mk}), plus G's entry.
 */
static void build_liouvillian(const orc_problem *p, cplx *L)
{
    const int N = p->N, NN = N * N;
    cplx *H = malloc((size_t)NN * sizeof(cplx));
    load_c(NN, p->H0, H);
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k)
            for (int l = 0; l < N; ++l)
                for (int m = 0; m < N; ++m) {
                    cplx v = 0;
                    if (k == m) v += H[j * N + l];
                    if (j == l) v -= H[m * N + k];
                    v *= -I / ORC_HBAR;
                    if (p->G) {
                        int idx = (j * N + k) * NN + (l * N + m);
                        v += p->G[2 * idx] + I * p->G[2 * idx + 1];
                    }
                    L[(j * N + k) * NN + (l * N + m)] = v;
                }
    free(H);
}

static void superop_apply(int NN, const cplx *S, const cplx *x, cplx *y)
{
    for (int r = 0; r < NN; ++r) {
        cplx s = 0;
        for (int c = 0; c < NN; ++c)
            s += S[r * NN + c] * x[c];
        y[r] = s;
    }
}

/* Tr{mu X} = sum_{j,k} mu_{jk} X_{kj}. */
static cplx trace_prod(int N, const cplx *mu, const cplx *X)
{
    cplx s = 0;
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k)
            s += mu[j * N + k] * X[k * N + j];
    return s;
}

/* --------------------------------------------------------- one-cell update */

typedef struct {
    int N;
    cplx *A0;   /* exp((L0 + G) dt/2), N^2 x N^2 */
    cplx *L;    /* L0 + G */
    cplx *mu;   /* N x N */
    double dt, N_a;
} cell_ops;

static int cell_ops_init(const orc_problem *p, cell_ops *ops)
{
    const int N = p->N, NN = N * N;
    ops->N = N;
    ops->dt = p->dt;
    ops->N_a = p->N_a;
    ops->A0 = malloc((size_t)NN * NN * sizeof(cplx));
    ops->L = malloc((size_t)NN * NN * sizeof(cplx));
    ops->mu = malloc((size_t)NN * sizeof(cplx));
    cplx *Ls = malloc((size_t)NN * NN * sizeof(cplx));
    if (!ops->A0 || !ops->L || !ops->mu || !Ls) {
        free(Ls);
        return -2;
    }
    build_liouvillian(p, ops->L);
    for (int i = 0; i < NN * NN; ++i)
        Ls[i] = ops->L[i] * (0.5 * p->dt);
    int rc = expm_c(NN, Ls, ops->A0);
    free(Ls);
    load_c(NN, p->mu, ops->mu);
    return rc;
}

static void cell_ops_free(cell_ops *ops)
{
    free(ops->A0); free(ops->L); free(ops->mu);
}

/*
 * One Strang step of one cell (Sec. 4.1, Eq. 23 read in rho-space):
 * rho' = A0(rho), rho'' = V rho' V^+ with V = exp(+i mu E dt / hbar),
 * rho^{n+1/2} = A0(rho''); returns dP/dt^{n+1/2} = N_a Tr{mu (L0+G)(rho^{n+1/2})}
 * (Eqs. 3 and 5). rho is N x N complex, updated in place.
 */
static int cell_step(const cell_ops *ops, cplx *rho, double E, double *dPdt)
{
    const int N = ops->N, NN = N * N;
    cplx r1[64], r2[64], V[64], Vh[64], T[64], arg[64];
    superop_apply(NN, ops->A0, rho, r1);
    for (int i = 0; i < NN; ++i)
        arg[i] = I * ops->mu[i] * (E * ops->dt / ORC_HBAR);
    int rc = expm_c(N, arg, V);
    if (rc)
        return rc;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            Vh[i * N + j] = conj(V[j * N + i]);
    mat_mul(N, V, r1, T);
    mat_mul(N, T, Vh, r2);
    superop_apply(NN, ops->A0, r2, rho);
    superop_apply(NN, ops->L, rho, r1);
    *dPdt = ops->N_a * creal(trace_prod(N, ops->mu, r1));
    return 0;
}

/*
 * Circulant kernel of the staggered spectral derivative on n points of spacing
 * dx: out_j = sum_i c[(j - i) mod n] in_i gives the derivative of the
 * trigonometric interpolant of in at the points shifted by half * dx
 * (half = +1/2: from E points to H points; -1/2: from H points to E points).
 * c[d] = (1/n) sum_m i k_m e^{i k_m half dx} e^{2 pi i m d / n}; the imaginary
 * parts cancel (the interpolant of real samples is real), so only the real
 * part is kept.
 */
static void spectral_kernel(long n, double dx, double half, double *c)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (long d = 0; d < n; ++d) {
        long double complex acc = 0.0L;
        for (long m = 0; m < n; ++m) {
            const long ms = (m <= n / 2) ? m : m - n;
            const double k = two_pi * (double)ms / ((double)n * dx);
            const long double complex mult = I * k * cexpl(I * (long double)(k * half * dx));
            acc += mult * cexpl(I * (long double)(two_pi * (double)((m * d) % n) / (double)n));
        }
        c[d] = (double)(creall(acc) / (long double)n);
    }
}

/* out_j = sum_i c[(j - i) mod n] in_i */
static void circulant_apply(long n, const double *c, const double *in, double *out)
{
    for (long j = 0; j < n; ++j) {
        double acc = 0.0;
        for (long i = 0; i < n; ++i)
            acc += c[((j - i) % n + n) % n] * in[i];
        out[j] = acc;
    }
}

/* ---------------------------------------------------------------- exported */

/* The staggered spectral derivative of n periodic samples (see above). */
int orc_spectral_derivative(long n, double dx, double half, const double *in, double *out)
{
    if (n < 2) return -1;
    double *c = malloc((size_t)n * sizeof(double));
    if (!c) return -2;
    spectral_kernel(n, dx, half, c);
    circulant_apply(n, c, in, out);
    free(c);
    return 0;
}

/* exp(A) of an n x n complex matrix (interleaved re/im, row-major). */
int orc_expm(int n, const double *A, double *X)
{
    size_t nn = (size_t)n * n;
    cplx *a = malloc(nn * sizeof(cplx)), *x = malloc(nn * sizeof(cplx));
    if (!a || !x) { free(a); free(x); return -2; }
    load_c(nn, A, a);
    int rc = expm_c(n, a, x);
    store_c(nn, x, X);
    free(a); free(x);
    return rc;
}

/* The matrix L0 + G (N^2 x N^2 complex) of the problem. */
int orc_liouvillian(const orc_problem *p, double *L)
{
    int NN = p->N * p->N;
    cplx *l = malloc((size_t)NN * NN * sizeof(cplx));
    if (!l) return -2;
    build_liouvillian(p, l);
    store_c((size_t)NN * NN, l, L);
    free(l);
    return 0;
}

/* dP/dt = N_a Tr{mu (L0 + G)(rho)} for one density matrix (Eqs. 3 and 5). */
int orc_dpdt(const orc_problem *p, const double *rho, double *out)
{
    const int N = p->N, NN = N * N;
    if (N < 2 || N > 8) return -1;
    cplx *L = malloc((size_t)NN * NN * sizeof(cplx));
    cplx r[64], y[64], mu[64];
    if (!L) return -2;
    build_liouvillian(p, L);
    load_c(NN, rho, r);
    load_c(NN, p->mu, mu);
    superop_apply(NN, L, r, y);
    *out = p->N_a * creal(trace_prod(N, mu, y));
    free(L);
    return 0;
}

/*
 * One medium cell driven by a prescribed field: for n = 0 .. n_steps-1 apply
 * the Strang step with E^n = E_seq[n]; dpdt[n] (if not NULL) receives
 * dP/dt^{n+1/2}. rho (N x N complex) is updated in place.
 */
int orc_cell(const orc_problem *p, double *rho, long n_steps, const double *E_seq, double *dpdt)
{
    const int N = p->N, NN = N * N;
    if (N < 2 || N > 8) return -1;
    cell_ops ops;
    int rc = cell_ops_init(p, &ops);
    if (rc) { cell_ops_free(&ops); return rc; }
    cplx r[64];
    load_c(NN, rho, r);
    for (long n = 0; n < n_steps && rc == 0; ++n) {
        double dp;
        rc = cell_step(&ops, r, E_seq[n], &dp);
        if (dpdt) dpdt[n] = dp;
    }
    store_c(NN, r, rho);
    cell_ops_free(&ops);
    return rc;
}

/*
 * The coupled solver. E (n_cells), H (n_cells; H[i] is H_y at i + 1/2) and rho
 * (n_medium x N x N complex) hold the state at E^n, H^{n-1/2}, rho^{n-1/2} and
 * are advanced in place by n_steps steps. src (n_steps samples) may be NULL.
 * If probe is not NULL, probe[n] receives E at probe_cell after step n.
 * threads <= 0 uses the OpenMP default.
 */
int orc_run(const orc_problem *p, double *E, double *H, double *rho, long n_steps,
            const double *src, long probe_cell, double *probe, int threads)
{
    const int N = p->N, NN = N * N;
    const long n = p->n_cells, mb = p->medium_begin, me = p->medium_end;
    if (N < 2 || N > 8 || n < 3 || mb < 0 || me < mb || me > n)
        return -1;
    const long nm = me - mb;
    const double eps = ORC_EPS0 * p->eps_r, muu = ORC_MU0 * p->mu_r;
    const double ch = p->dt / (muu * p->dx);
    const double sg = p->sigma * p->dt / (2.0 * eps);
    const double ca = (1.0 - sg) / (1.0 + sg);
    const double cb = (p->dt / eps) / (1.0 + sg);
    const double cv = 1.0 / sqrt(eps * muu);
    const double kappa = (cv * p->dt - p->dx) / (cv * p->dt + p->dx);

    cell_ops ops;
    int rc = cell_ops_init(p, &ops);
    if (rc) { cell_ops_free(&ops); return rc; }

    const int pstd = p->maxwell == ORC_PSTD;
    if (pstd && p->boundary != ORC_BC_PERIODIC) { cell_ops_free(&ops); return -1; }
    cplx *r = malloc((size_t)(nm > 0 ? nm : 1) * NN * sizeof(cplx));
    double *dP = calloc((size_t)n, sizeof(double));
    double *En = malloc((size_t)n * sizeof(double));
    double *cp = pstd ? malloc((size_t)n * sizeof(double)) : NULL;
    double *cm = pstd ? malloc((size_t)n * sizeof(double)) : NULL;
    double *dv = pstd ? malloc((size_t)n * sizeof(double)) : NULL;
    if (!r || !dP || !En || (pstd && (!cp || !cm || !dv))) {
        free(r); free(dP); free(En); free(cp); free(cm); free(dv); cell_ops_free(&ops); return -2;
    }
    if (pstd) {
        spectral_kernel(n, p->dx, 0.5, cp);
        spectral_kernel(n, p->dx, -0.5, cm);
    }
    load_c((size_t)nm * NN, rho, r);

#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#else
    (void)threads;
#endif

    for (long step = 0; step < n_steps && rc == 0; ++step) {
        /* H^{n+1/2} from E^n (Eq. 1b on the staggered grid of Fig. 1) */
        if (pstd) {
            circulant_apply(n, cp, E, dv);
            for (long i = 0; i < n; ++i)
                H[i] += (p->dt / muu) * dv[i];
        } else if (p->boundary == ORC_BC_PERIODIC) {
            for (long i = 0; i < n; ++i)
                H[i] += ch * (E[(i + 1) % n] - E[i]);
        } else {
            for (long i = 0; i < n - 1; ++i)
                H[i] += ch * (E[i + 1] - E[i]);
        }

        /* rho^{n-1/2} -> rho^{n+1/2} with E^n, and dP/dt^{n+1/2} (Eq. 23, Eq. 5) */
        int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
        for (long m = 0; m < nm; ++m) {
            double dp = 0.0;
            if (cell_step(&ops, r + m * NN, E[mb + m], &dp))
                bad |= 1;
            dP[mb + m] = dp;
        }
        if (bad) { rc = -3; break; }

        /* E^{n+1} from H^{n+1/2} and dP/dt^{n+1/2} (Eq. 1a) */
        if (pstd) {
            circulant_apply(n, cm, H, dv);
            for (long i = 0; i < n; ++i)
                En[i] = ca * E[i] + cb * (dv[i] - dP[i]);
        } else {
            for (long i = 0; i < n; ++i) {
                long im1 = (i == 0) ? n - 1 : i - 1;
                En[i] = ca * E[i] + cb * ((H[i] - H[im1]) / p->dx - dP[i]);
            }
        }
        if (p->boundary == ORC_BC_OPEN) {
            En[0] = E[0];
            En[n - 1] = E[n - 2] + kappa * (En[n - 2] - E[n - 1]);
        } else if (p->boundary == ORC_BC_WINDOW) {
            En[0] = E[0];
            En[n - 1] = E[n - 1];
        }
        if (src && p->source_kind == ORC_SRC_HARD)
            En[p->source_cell] = src[step];
        else if (src && p->source_kind == ORC_SRC_SOFT)
            En[p->source_cell] += src[step];
        memcpy(E, En, (size_t)n * sizeof(double));
        if (probe)
            probe[step] = E[probe_cell];
    }
    store_c((size_t)nm * NN, r, rho);
    free(r); free(dP); free(En); free(cp); free(cm); free(dv);
    cell_ops_free(&ops);
    return rc;
}
