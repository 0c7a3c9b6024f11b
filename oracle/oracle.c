/*
 * oracle.c -- plain CPU FP64 oracle of the NFFT nonlocal-denoising hot path.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may load or call this library.  It shares no
 * code, header, table or helper with the CUDA library; it computes the
 * method's *definition* (direct O(N^2) kernel sums) and the paper's solvers
 * in the paper's own coordinates, slowly and in double precision.
 *
 * Notation follows the paper (arXiv 2407.06834):
 *   f   noisy image, n = n1 n2 pixels (Sec. 2.3, Sec. 5)
 *   W_l feature windows, L of them (Eq. (2.8) continuous_ANOVA, Sec. 5)
 *   Gamma  ANOVA kernel with zero diagonal (Eq. discrete_ANOVA + the
 *          zero-diagonal convention that follows it)
 *   eta = Gamma 1,  L = diag(eta) - Gamma,  A = lambda I + mu L
 *          (Eq. discretized-state, Sec. 4.2)
 *   U   Helmert change of basis for v = 1 (Eq. ULap)
 *   P_a = lambda I + mu diag(eta)  (Sec. 4.3.1)
 *
 * Every function below cites the passage it follows.  No blocking, fusion or
 * reordering beyond the stated definitions; OpenMP only splits independent
 * rows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Features and windows                                                      */
/* ------------------------------------------------------------------------ */

/* Mirror an out-of-range index into [0, n) without repeating the edge pixel
 * ("reflect" padding: -1 -> 1, n -> n-2). */
static int reflect_index(int i, int n)
{
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

/* Patch features, Sec. 5: for every pixel a closed square patch of radius rho
 * of the noisy image, giving n x (2 rho + 1)^2 features.  Pixel i = r n2 + c
 * (row-major), patch dim k = (dr + rho)(2 rho + 1) + (dc + rho).
 * pad = 0: zero padding (the paper's choice); pad = 1: reflect padding. */
void orc_patch_features(const double *img, int n1, int n2, int rho, int pad,
                        double *feat)
{
    int P = 2 * rho + 1, D = P * P;
    for (int r = 0; r < n1; ++r)
        for (int c = 0; c < n2; ++c) {
            double *out = feat + ((long)r * n2 + c) * D;
            for (int dr = -rho; dr <= rho; ++dr)
                for (int dc = -rho; dc <= rho; ++dc) {
                    int rr = r + dr, cc = c + dc, k = (dr + rho) * P + (dc + rho);
                    double val;
                    if (pad == 0) {
                        val = (rr < 0 || rr >= n1 || cc < 0 || cc >= n2)
                                  ? 0.0 : img[(long)rr * n2 + cc];
                    } else {
                        val = img[(long)reflect_index(rr, n1) * n2 +
                                  reflect_index(cc, n2)];
                    }
                    out[k] = val;
                }
        }
}

/* Window coordinates W_l[f]_i (Eq. discrete_ANOVA): window l picks the
 * feature dims win[3l..3l+2]; an entry -1 is a zero-valued dimension.
 * Output layout: coords[(l N + i) 3 + t]. */
void orc_window_coords(const double *feat, long N, int D, int L,
                       const int *win, double *coords)
{
    for (int l = 0; l < L; ++l)
        for (long i = 0; i < N; ++i)
            for (int t = 0; t < 3; ++t) {
                int d = win[3 * l + t];
                coords[((long)l * N + i) * 3 + t] =
                    (d < 0) ? 0.0 : feat[i * (long)D + d];
            }
}

/* ------------------------------------------------------------------------ */
/* Kernel sums (definition)                                                  */
/* ------------------------------------------------------------------------ */

/* One ANOVA kernel entry, Eq. discrete_ANOVA:
 * gamma_ij = (1/L) sum_l exp(-sigma^-2 ||W_l[f]_i - W_l[f]_j||^2). */
static double anova_entry(const double *coords, long N, int L, double inv_s2,
                          long i, long j)
{
    double acc = 0.0;
    for (int l = 0; l < L; ++l) {
        const double *ci = coords + ((long)l * N + i) * 3;
        const double *cj = coords + ((long)l * N + j) * 3;
        double d0 = ci[0] - cj[0], d1 = ci[1] - cj[1], d2 = ci[2] - cj[2];
        acc += exp(-inv_s2 * (d0 * d0 + d1 * d1 + d2 * d2));
    }
    return acc / L;
}

/* y = Gamma_full v for the listed rows, where Gamma_full keeps the diagonal
 * gamma_ii = 1 (the fast summation of Sec. 3 sums over all j, including
 * j = i).  rows == NULL means all N rows, y indexed like v. */
void orc_gamma_full_rows(const double *coords, long N, int L, double sigma,
                         const double *v, const long *rows, long nrows,
                         double *y)
{
    double inv_s2 = 1.0 / (sigma * sigma);
    long nr = rows ? nrows : N;
#pragma omp parallel for schedule(dynamic, 16)
    for (long r = 0; r < nr; ++r) {
        long i = rows ? rows[r] : r;
        double acc = 0.0;
        for (long j = 0; j < N; ++j)
            acc += anova_entry(coords, N, L, inv_s2, i, j) * v[j];
        y[r] = acc;
    }
}

void orc_gamma_full_matvec(const double *coords, long N, int L, double sigma,
                           const double *v, double *y)
{
    orc_gamma_full_rows(coords, N, L, sigma, v, NULL, 0, y);
}

/* y = Gamma v with the zero diagonal of Sec. 2.3: the j = i term is left out
 * because it cancels in the Laplacian. */
void orc_gamma_matvec(const double *coords, long N, int L, double sigma,
                      const double *v, double *y)
{
    double inv_s2 = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < N; ++i) {
        double acc = 0.0;
        for (long j = 0; j < N; ++j)
            if (j != i) acc += anova_entry(coords, N, L, inv_s2, i, j) * v[j];
        y[i] = acc;
    }
}

/* Dense Gamma (zero diagonal), row-major N x N, for small-N spectral tests. */
void orc_gamma_dense(const double *coords, long N, int L, double sigma,
                     double *G)
{
    double inv_s2 = 1.0 / (sigma * sigma);
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < N; ++i)
        for (long j = 0; j < N; ++j)
            G[i * N + j] = (i == j) ? 0.0 : anova_entry(coords, N, L, inv_s2, i, j);
}

/* Degrees eta = Gamma 1 (Sec. 2.3, eta^h := Gamma^h 1). */
void orc_degrees(const double *coords, long N, int L, double sigma, double *eta)
{
    double *ones = (double *)malloc(sizeof(double) * N);
    for (long i = 0; i < N; ++i) ones[i] = 1.0;
    orc_gamma_matvec(coords, N, L, sigma, ones, eta);
    free(ones);
}

/* The diagonal preconditioner P_b' of Sec. 4.3.3 (Eq. ANOVA_Norm_2_Prec):
 *   (P_b')_ii^2 = (mu / L)^2 sum_l sum_{j != i} exp(-2 sigma^-2 ||W_l[f]_i - W_l[f]_j||^2)
 *                 + (lambda + mu eta_i)^2,
 * i.e. the first L (per-window) terms of the Pascal-simplex expansion of
 * (Gamma o Gamma) 1 added to the square of P_a = lambda + mu eta. */
void orc_pb_diag(const double *coords, long N, int L, double sigma, double lambda,
                 double mu, double *P)
{
    double *eta = (double *)malloc(sizeof(double) * N);
    orc_degrees(coords, N, L, sigma, eta);
    double two_inv_s2 = 2.0 / (sigma * sigma);
    double w = (mu / L) * (mu / L);
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int l = 0; l < L; ++l) {
            const double *ci = coords + ((long)l * N + i) * 3;
            for (long j = 0; j < N; ++j) {
                if (j == i) continue;
                const double *cj = coords + ((long)l * N + j) * 3;
                double d0 = ci[0] - cj[0], d1 = ci[1] - cj[1], d2 = ci[2] - cj[2];
                acc += exp(-two_inv_s2 * (d0 * d0 + d1 * d1 + d2 * d2));
            }
        }
        double pa = lambda + mu * eta[i];
        P[i] = sqrt(w * acc + pa * pa);
    }
    free(eta);
}

/* y = A v = lambda v + mu (diag(eta) - Gamma) v, Eq. discretized-state. */
void orc_A_apply(const double *coords, long N, int L, double sigma,
                 double lambda, double mu, const double *eta,
                 const double *v, double *y)
{
    double *gv = (double *)malloc(sizeof(double) * N);
    orc_gamma_matvec(coords, N, L, sigma, v, gv);
    for (long i = 0; i < N; ++i)
        y[i] = lambda * v[i] + mu * (eta[i] * v[i] - gv[i]);
    free(gv);
}

/* ------------------------------------------------------------------------ */
/* Truncated Fourier series of the Gaussian (fast-summation target, Sec. 3)  */
/* ------------------------------------------------------------------------ */

/* Fourier transform of exp(-t^2 / s^2) at frequency k:
 * int exp(-t^2/s^2) exp(-2 pi i k t) dt = sqrt(pi) s exp(-pi^2 s^2 k^2).
 * These are the coefficients the FGT of Sec. 3 multiplies by. */
double orc_gauss_fourier_coeff(double s, double k)
{
    return sqrt(M_PI) * s * exp(-M_PI * M_PI * s * s * k * k);
}

/* K_M(t) = sum_{|k| < M/2} ghat(k) e^{2 pi i k t}: the bandlimited,
 * 1-periodic approximation of exp(-t^2/s^2) that the NFFT-based FGT
 * evaluates (Eq. NFFT with I_M, multiplied by the Gaussian coefficients). */
double orc_trig_kernel_1d(double t, double s, int M)
{
    double acc = orc_gauss_fourier_coeff(s, 0.0);
    for (int k = 1; 2 * k < M; ++k)
        acc += 2.0 * orc_gauss_fourier_coeff(s, (double)k) * cos(2.0 * M_PI * k * t);
    return acc;
}

/* Affine map of the window coordinates onto the torus:
 * x~ = s (x - c_l), c_l the per-window, per-dim midrange, s = fill / R with
 * R the largest per-dim coordinate range over all windows (R := 1 when all
 * coordinates coincide).  Returns s. */
double orc_torus_map(const double *coords, long N, int L, double fill,
                     double *tcoords)
{
    double R = 0.0;
    double *ctr = (double *)malloc(sizeof(double) * 3 * L);
    for (int l = 0; l < L; ++l)
        for (int t = 0; t < 3; ++t) {
            double lo = coords[((long)l * N) * 3 + t], hi = lo;
            for (long i = 0; i < N; ++i) {
                double x = coords[((long)l * N + i) * 3 + t];
                if (x < lo) lo = x;
                if (x > hi) hi = x;
            }
            ctr[3 * l + t] = 0.5 * (lo + hi);
            if (hi - lo > R) R = hi - lo;
        }
    if (!(R > 0.0)) R = 1.0;
    double s = fill / R;
    for (int l = 0; l < L; ++l)
        for (long i = 0; i < N; ++i)
            for (int t = 0; t < 3; ++t)
                tcoords[((long)l * N + i) * 3 + t] =
                    s * (coords[((long)l * N + i) * 3 + t] - ctr[3 * l + t]);
    free(ctr);
    return s;
}

/* y_i = (1/L) sum_l sum_j v_j prod_{d=1..3} K_M(x~_li,d - x~_lj,d):
 * the fast summation's target with the Gaussian replaced by its truncated
 * Fourier series, diagonal kept (Sec. 3).  sigma_s = s sigma is the kernel
 * width on the torus. */
void orc_trig_full_matvec(const double *tcoords, long N, int L,
                          double sigma_s, int M, const double *v, double *y)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (long i = 0; i < N; ++i) {
        double acc = 0.0;
        for (long j = 0; j < N; ++j) {
            double e = 0.0;
            for (int l = 0; l < L; ++l) {
                const double *ci = tcoords + ((long)l * N + i) * 3;
                const double *cj = tcoords + ((long)l * N + j) * 3;
                e += orc_trig_kernel_1d(ci[0] - cj[0], sigma_s, M) *
                     orc_trig_kernel_1d(ci[1] - cj[1], sigma_s, M) *
                     orc_trig_kernel_1d(ci[2] - cj[2], sigma_s, M);
            }
            acc += e * v[j];
        }
        y[i] = acc / L;
    }
}

/* ------------------------------------------------------------------------ */
/* Helmert change of basis U (Eq. ULap, the v = 1 case of Eq.               */
/* UnitaryGeneralForm): column 1 = 1/sqrt(n); column i >= 2 =               */
/* (1, ..., 1, -(i-1), 0, ..., 0) / sqrt(i (i-1)).  Both actions are O(n)   */
/* shifted cumulative sums, as the paper's SCS formulas state.              */
/* ------------------------------------------------------------------------ */

/* u = U x: u_j = x_1/sqrt(n) + sum_{i>j} x_i / sqrt(i(i-1)) - x_j sqrt((j-1)/j)
 * (1-based j; the last term is absent for j = 1). */
void orc_U_apply(const double *x, long n, double *u)
{
    double tail = 0.0;                    /* sum_{i > j} x_i b_i */
    double head = x[0] / sqrt((double)n);
    for (long j = n; j >= 1; --j) {
        double uj = head + tail;
        if (j >= 2) uj -= x[j - 1] * sqrt((double)(j - 1) / (double)j);
        u[j - 1] = uj;
        if (j >= 2) tail += x[j - 1] / sqrt((double)j * (double)(j - 1));
    }
}

/* g = U^T x: g_1 = sum_j x_j / sqrt(n); for i >= 2
 * g_i = (sum_{j<i} x_j - (i-1) x_i) / sqrt(i(i-1)). */
void orc_Ut_apply(const double *x, long n, double *g)
{
    double total = 0.0;
    for (long j = 0; j < n; ++j) total += x[j];
    g[0] = total / sqrt((double)n);
    double prefix = x[0];                 /* sum_{j < i} x_j */
    for (long i = 2; i <= n; ++i) {
        g[i - 1] = (prefix - (double)(i - 1) * x[i - 1]) /
                   sqrt((double)i * (double)(i - 1));
        prefix += x[i - 1];
    }
}

/* ------------------------------------------------------------------------ */
/* Solvers                                                                    */
/* ------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

typedef struct {
    const double *coords;
    long N;
    int L;
    double sigma, lambda, mu;
    const double *eta;   /* Gamma 1 */
    const double *P;     /* diagonal of P_a, or NULL for no preconditioner */
    double *w1, *w2;     /* length-N scratch */
} orc_sys;

/* q = B2 p with B2 = pi_2(U^T A U) (Sec. 4.1 and Sec. 4.3.2): lift p to
 * (0, p), map by U, apply A, map back by U^T and drop the first entry. */
static void block2_apply(orc_sys *S, const double *p, double *q)
{
    long N = S->N;
    S->w1[0] = 0.0;
    memcpy(S->w1 + 1, p, sizeof(double) * (N - 1));
    orc_U_apply(S->w1, N, S->w2);
    orc_A_apply(S->coords, N, S->L, S->sigma, S->lambda, S->mu, S->eta,
                S->w2, S->w1);
    orc_Ut_apply(S->w1, N, S->w2);
    memcpy(q, S->w2 + 1, sizeof(double) * (N - 1));
}

/* z = pi_2(U^T P^-1 U) r, the projected ("dense") preconditioner
 * P_{U,P}^{-1} of Sec. 4.3.2 restricted to the second block. */
static void block2_prec(orc_sys *S, const double *r, double *z)
{
    long N = S->N;
    if (!S->P) { memcpy(z, r, sizeof(double) * (N - 1)); return; }
    S->w1[0] = 0.0;
    memcpy(S->w1 + 1, r, sizeof(double) * (N - 1));
    orc_U_apply(S->w1, N, S->w2);
    for (long i = 0; i < N; ++i) S->w2[i] /= S->P[i];
    orc_Ut_apply(S->w2, N, S->w1);
    memcpy(z, S->w1 + 1, sizeof(double) * (N - 1));
}

/* Deflated (decoupled) CG of Sec. 4.1 / Sec. 4.3.2 / Sec. 5.4, in the
 * paper's coordinates: g = U^T b, x_1 = g_1 / lambda, CG on
 * B2 x_{2:n} = g_{2:n} preconditioned by pi_2(U^T P_a^-1 U) (precond = 1,
 * "P_{U,a}"), by pi_2(U^T P_b'^-1 U) (precond = 2, P_b' of Sec. 4.3.3) or
 * unpreconditioned (precond = 0, "I_U"); then u = U x.
 * Stops when ||r|| <= tol ||b|| (r the CG residual of the second block,
 * whose norm equals ||b - A u|| because U is orthogonal and the first block
 * is solved exactly).  hist[k] = ||r_k|| / ||b|| for k = 0..iters.
 * Returns 0 converged, 1 not converged within maxit, -4 breakdown. */
int orc_pcg_deflated(const double *coords, long N, int L, double sigma,
                     double lambda, double mu, const double *b, double tol,
                     int maxit, int precond, double *u, double *hist,
                     int *iters)
{
    double *eta = (double *)malloc(sizeof(double) * N);
    double *P = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    double *x = (double *)calloc(N, sizeof(double));
    long n2 = N - 1;
    double *r = (double *)malloc(sizeof(double) * (n2 + 1));
    double *z = (double *)malloc(sizeof(double) * (n2 + 1));
    double *p = (double *)malloc(sizeof(double) * (n2 + 1));
    double *q = (double *)malloc(sizeof(double) * (n2 + 1));
    orc_sys S = {coords, N, L, sigma, lambda, mu, eta, NULL,
                 (double *)malloc(sizeof(double) * N),
                 (double *)malloc(sizeof(double) * N)};
    orc_degrees(coords, N, L, sigma, eta);
    if (precond == 2)
        orc_pb_diag(coords, N, L, sigma, lambda, mu, P);
    else
        for (long i = 0; i < N; ++i) P[i] = lambda + mu * eta[i];
    if (precond) S.P = P;

    orc_Ut_apply(b, N, g);
    x[0] = g[0] / lambda;                 /* first block solved exactly */
    double bnorm = sqrt(dot(b, b, N));
    if (bnorm == 0.0) bnorm = 1.0;
    double *y = x + 1;                    /* second-block unknowns, start 0 */
    memcpy(r, g + 1, sizeof(double) * n2);
    int status = 1, k = 0;
    hist[0] = sqrt(dot(r, r, n2)) / bnorm;
    if (n2 == 0 || hist[0] <= tol) status = 0;
    if (status != 0) {
        block2_prec(&S, r, z);
        memcpy(p, z, sizeof(double) * n2);
        double rz = dot(r, z, n2);
        for (k = 1; k <= maxit; ++k) {
            block2_apply(&S, p, q);
            double pq = dot(p, q, n2);
            if (!(pq > 0.0) || !isfinite(pq)) { status = -4; --k; break; }
            double a = rz / pq;
            for (long i = 0; i < n2; ++i) { y[i] += a * p[i]; r[i] -= a * q[i]; }
            hist[k] = sqrt(dot(r, r, n2)) / bnorm;
            if (hist[k] <= tol) { status = 0; break; }
            block2_prec(&S, r, z);
            double rz_new = dot(r, z, n2);
            double beta = rz_new / rz;
            rz = rz_new;
            for (long i = 0; i < n2; ++i) p[i] = z[i] + beta * p[i];
        }
        if (k > maxit) k = maxit;
    }
    *iters = k;
    orc_U_apply(x, N, u);
    free(eta); free(P); free(g); free(x); free(r); free(z); free(p); free(q);
    free(S.w1); free(S.w2);
    return status;
}

/* CG / Jacobi-PCG in the original basis (Sec. 5.3, Table 2 with no
 * preconditioner and x0 = f; Sec. 5.4 "P_a"): precond 0 = I, 1 = P_a,
 * 2 = P_b' (Sec. 4.3.3).
 * x0 may be NULL (zero start).  Same stopping rule and history as above. */
int orc_cg(const double *coords, long N, int L, double sigma, double lambda,
           double mu, const double *b, const double *x0, double tol, int maxit,
           int precond, double *u, double *hist, int *iters)
{
    double *eta = (double *)malloc(sizeof(double) * N);
    double *P = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N);
    double *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    orc_degrees(coords, N, L, sigma, eta);
    if (precond == 2)
        orc_pb_diag(coords, N, L, sigma, lambda, mu, P);
    else
        for (long i = 0; i < N; ++i) P[i] = lambda + mu * eta[i];
    for (long i = 0; i < N; ++i) u[i] = x0 ? x0[i] : 0.0;
    orc_A_apply(coords, N, L, sigma, lambda, mu, eta, u, q);
    for (long i = 0; i < N; ++i) r[i] = b[i] - q[i];
    double bnorm = sqrt(dot(b, b, N));
    if (bnorm == 0.0) bnorm = 1.0;
    int status = 1, k = 0;
    hist[0] = sqrt(dot(r, r, N)) / bnorm;
    if (hist[0] <= tol) status = 0;
    if (status != 0) {
        for (long i = 0; i < N; ++i) z[i] = precond ? r[i] / P[i] : r[i];
        memcpy(p, z, sizeof(double) * N);
        double rz = dot(r, z, N);
        for (k = 1; k <= maxit; ++k) {
            orc_A_apply(coords, N, L, sigma, lambda, mu, eta, p, q);
            double pq = dot(p, q, N);
            if (!(pq > 0.0) || !isfinite(pq)) { status = -4; --k; break; }
            double a = rz / pq;
            for (long i = 0; i < N; ++i) { u[i] += a * p[i]; r[i] -= a * q[i]; }
            hist[k] = sqrt(dot(r, r, N)) / bnorm;
            if (hist[k] <= tol) { status = 0; break; }
            for (long i = 0; i < N; ++i) z[i] = precond ? r[i] / P[i] : r[i];
            double rz_new = dot(r, z, N);
            double beta = rz_new / rz;
            rz = rz_new;
            for (long i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
        }
        if (k > maxit) k = maxit;
    }
    *iters = k;
    free(eta); free(P); free(r); free(z); free(p); free(q);
    return status;
}
