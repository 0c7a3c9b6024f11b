/*
 * nlh.h -- C ABI of the GB300 (sm_103a) NFFT nonlocal-denoising library.
 *
 * The library solves the nonlocal system of arXiv 2407.06834
 *     (lambda I + mu L) u = b,   L = diag(eta) - Gamma,   eta = Gamma 1
 * (Eq. discretized-state, Sec. 4.2) matrix-free.  Gamma is the unnormalised
 * extended Gaussian ANOVA kernel over per-pixel patch features
 * (Eq. discrete_ANOVA, with the zero diagonal of Sec. 2.3), and every
 * product with Gamma is an NFFT fast Gauss transform per feature window
 * (Sec. 3).  Throughout, mu = 1 and alpha = lambda / mu, so the system is
 * (alpha I + L) u = b; the denoising right-hand side is b = alpha f.
 *
 * Conventions for every entry point:
 *   - Vectors and feature matrices are DEVICE pointers owned by the caller;
 *     the library never frees or keeps them beyond the call.  All FP64.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; a call that returns host-visible
 *     results (plan creation, solve info) synchronises that stream only.
 *   - Errors come back as nlh_status codes, never as exceptions or aborts;
 *     nlh_last_error() gives a message for the calling thread.
 *   - The library owns everything inside a plan (grids, permutations,
 *     tables, solver workspace); nlh_plan_destroy frees it.
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef NLH_H
#define NLH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NLH_OK = 0,
    NLH_ERR_NOT_CONVERGED = 1, /* warning: u holds the last iterate         */
    NLH_ERR_ARG = -1,          /* invalid argument (message says which)     */
    NLH_ERR_CUDA = -2,         /* a CUDA runtime call failed                */
    NLH_ERR_OOM = -3,          /* device allocation failed                  */
    NLH_ERR_BREAKDOWN = -4,    /* CG breakdown: p^T A p <= 0 or not finite  */
    NLH_ERR_TIMEOUT = -5       /* a bounded device wait gave up             */
} nlh_status;

typedef struct nlh_plan_s *nlh_plan;

/* Sum over ranks of a plan that holds a range of the windows (Sec. 3: the
 * ANOVA kernel is the mean of L independent per-window Gauss transforms, so
 * ranks holding disjoint window ranges each compute a share of
 * Gamma_full x and one sum over the ranks completes it).  Called on the
 * host, at enqueue time, with the device FP64 vector buf of length n and
 * the stream of the current call; it must enqueue on that stream an
 * in-place sum of buf over all ranks (e.g. an NCCL all-reduce) and return.
 * ctx is the plan description's reduce_ctx. */
typedef void (*nlh_reduce_fn)(double *buf, int64_t n, void *stream, void *ctx);

/* NFFT arithmetic of a matvec.  NLH_DF32 carries every value as an
 * unevaluated sum of two floats (about 46-48 significant bits) so that the
 * FP64-accurate operator runs on the FP32 pipes; its grids and FFTs are FP64. */
enum { NLH_FP64 = 0, NLH_FP32 = 1, NLH_DF32 = 2 };

/* Patch features, Sec. 5: for every pixel the closed square patch of radius
 * `radius` of the image, zero padded (pad = 0, the paper's choice) or
 * reflect padded (pad = 1: index -1 maps to 1, n to n-2).
 *   image     device, n1 x n2 FP64, row-major (pixel i = r n2 + c)
 *   features  device, (n1 n2) x D FP64 with D = (2 radius + 1)^2, row-major;
 *             patch dim k = (dr + radius)(2 radius + 1) + (dc + radius).
 * Errors: NLH_ERR_ARG for n1, n2 < 1, radius < 0 or NULL pointers. */
nlh_status nlh_patch_features(const double *image, int n1, int n2, int radius,
                              int pad, double *features, void *stream);

/* Plan description.  Window l uses feature dims windows[3l .. 3l+2]
 * (Eq. continuous_ANOVA; windows of at most three dims, Sec. 3); an entry -1
 * is a zero-valued dim.  The Gaussian exp(-||x - y||^2 / sigma^2) of each
 * window is summed by an NFFT with bandwidth M per dim (frequencies
 * |k| < M/2), an oversampled grid of n_os points per dim and a Kaiser-Bessel
 * window that touches 2m grid points per dim. */
typedef struct {
    int64_t N;              /* points (pixels), >= 2                         */
    int D;                  /* feature dims per point, >= 1                  */
    int L;                  /* windows, 1..64                                */
    const int32_t *windows; /* HOST, L x 3 dim indices in [-1, D)            */
    double sigma;           /* kernel width, > 0                             */
    int M;                  /* even, 4 <= M <= n_os                          */
    int n_os;               /* power of two, 32..256                         */
    int m;                  /* 2..8, and 2m < n_os (0 with nfft_eps: auto)   */
    int precision;          /* bit 0: FP64 path, bit 1: FP32 path,
                               bit 2: double-float path (NLH_DF32)           */
    double torus_fill;      /* in (0, 1): fraction of the torus the points
                               span per dim; 0 = choose automatically        */
    int max_items_pts;      /* points per work item, 0 = default (64)        */
    double nfft_eps;        /* > 0: choose torus_fill, M and n_os (and m when
                               m = 0) so that the a-priori per-dim alias,
                               truncation and window errors are <= nfft_eps,
                               taking among the admissible grid sizes the one
                               with the least estimated work (a smaller grid
                               and a larger m for few points per cell);
                               M, n_os, torus_fill are then ignored          */
    int unit_points;        /* points per work unit (one CTA), 0 = 512       */
    int team[3];            /* launch shape of the spreading kernel per NFFT
                               arithmetic (index NLH_FP64, NLH_FP32,
                               NLH_DF32): 0 default, 1 and 2 the
                               alternatives compiled for 2m = 8 and 12;
                               other combinations use 0.  Results equal up
                               to the arithmetic's rounding                 */
    int window_first;       /* with window_count > 0: the plan holds windows */
    int window_count;       /* window_first .. window_first + window_count - 1
                               of the L listed (0: all).  The torus map is
                               taken over all L windows and sums are
                               normalised by L, so plans of complementary
                               ranges add up to the plan of all windows      */
    nlh_reduce_fn reduce;   /* range plans: NULL, or the sum over ranks.
                               With it every op of nlh_matvec, the degrees
                               and the solves are those of all L windows
                               (their Krylov loops are then host-driven,
                               checking every 4 iterations, since the
                               callback runs when a matvec is issued);
                               without it only op 0 (the range's share of
                               Gamma_full x) is defined                      */
    void *reduce_ctx;       /* passed to reduce                              */
    const double *image;    /* device n1 x n2 FP64 image the features are the
                               patches of (nlh_patch_features with
                               patch_radius, patch_pad; D = (2 r + 1)^2,
                               N = n1 n2), or NULL.  With it the plan keeps a
                               copy of the image instead of every point's
                               cell offsets, and the NFFT kernels recompute
                               each point's torus coordinates from the image
                               (FP64 arithmetic for the FP64 and
                               double-float paths, double-float for FP32):
                               12 B (FP32) or 24 B per point-window less
                               memory and traffic, at the cost of the
                               recomputation (measured 3-21 % slower
                               kernels: they are bound by arithmetic, not
                               by DRAM).  The caller guarantees that
                               features are those patches                 */
    int image_n1, image_n2; /* image rows, columns                           */
    int patch_radius;       /* >= 0                                          */
    int patch_pad;          /* 0 zero, 1 reflect (as nlh_patch_features)     */
} nlh_plan_desc;

/* Build a plan from a feature matrix (Sec. 3 / Sec. 5): window coordinates,
 * the affine map onto the torus x~ = s (x - c_l) with c_l the per-window
 * midrange and s = torus_fill / (largest per-dim range), the sort of the
 * points by grid cell with each point's offset inside its cell (the window
 * weights are evaluated from it in every matvec; with desc->image the
 * offsets are recomputed from the image instead of stored), the Fourier
 * multiplier tables and the degrees d = Gamma_full 1 (one matvec per
 * precision built).
 *   features  device, N x D FP64 row-major (e.g. from nlh_patch_features).
 * Synchronises `stream`.  Errors: NLH_ERR_ARG, NLH_ERR_OOM, NLH_ERR_CUDA. */
nlh_status nlh_plan_create(nlh_plan *out, const nlh_plan_desc *desc,
                           const double *features, void *stream);

/* Change sigma: recompute the multiplier tables and the degrees (Sec. 5.5
 * learns over sigma through theta = sigma^-2).  The torus map is kept.
 * Synchronises `stream`. */
nlh_status nlh_plan_set_sigma(nlh_plan plan, double sigma, void *stream);

typedef struct {
    int64_t N;
    int L, M, n_os, m, precision;
    double sigma, torus_fill, scale; /* scale s of the torus map             */
    double sigma_torus;              /* s * sigma                            */
    double max_range;                /* R, largest per-dim coordinate range  */
    int64_t n_items;                 /* work items over all windows          */
    int64_t occupied_cells;          /* non-empty (window, cell) pairs       */
    double est_trunc_err, est_alias_err; /* a-priori per-dim error estimates */
    int64_t device_bytes;            /* device memory owned by the plan      */
    int64_t n_units;                 /* work units (one CTA each)            */
    int max_items_pts, unit_points;  /* current tiling of the work           */
    int team[3];                     /* current launch shapes (see desc)     */
    int window_first, window_count;  /* the plan's window range              */
    int coords_from_image;           /* 1: coordinates recomputed from the
                                        image (desc.image), 0: stored        */
} nlh_plan_info;

nlh_status nlh_plan_get_info(nlh_plan plan, nlh_plan_info *info);

/* Re-split the plan's sorted points into work items of at most
 * max_items_pts points (all of one grid cell) and work units of at most
 * unit_points points (one CTA each), in place.  Changes only the
 * decomposition of the work, never the result beyond rounding.  The
 * degrees are recomputed in the new summation order (so that L 1 = 0 holds
 * to rounding), cached solve graphs are dropped and recaptured by the next
 * solve.  Synchronises `stream`. */
nlh_status nlh_plan_retile(nlh_plan plan, int max_items_pts, int unit_points, void *stream);

/* Set the launch shape (0..2; see nlh_plan_desc.team) of the spreading
 * kernel of one NFFT arithmetic (NLH_FP64, NLH_FP32, NLH_DF32).  Changes no
 * result beyond rounding.  A change of shape drops the cached solve graphs
 * and recomputes the degrees on the stream of the plan's last call, which it
 * synchronises. */
nlh_status nlh_plan_set_team(nlh_plan plan, int arith, int shape);

/* Autotuner: time `reps` matvecs (0 = 3) of every NFFT arithmetic in the
 * bit mask `precisions` (0 = all the plan built) for each tiling of a fixed
 * grid (max_items_pts in {32, 64, 128, 256} x unit_points in {256, 512, 1024,
 * 2048}) and, per arithmetic, each launch shape; leave the plan in the
 * tiling with the smallest sum over the arithmetics of their fastest shape,
 * with those shapes; report it (any output pointer may be NULL; best_team
 * has 3 entries indexed like nlh_plan_desc.team) and its summed matvec time
 * in ms.  Like nlh_plan_retile it recomputes the degrees and drops cached
 * solve graphs.  Synchronises `stream`. */
nlh_status nlh_plan_autotune(nlh_plan plan, int precisions, int reps, int *best_kmax,
                             int *best_unit_points, int *best_team, double *best_ms,
                             void *stream);

/* Matrix-free products (Sec. 3 and Eq. discretized-state), y and x device
 * FP64 vectors of length N (y must not alias x):
 *   op 0: y = Gamma_full x          (kernel sum over all j, diagonal kept)
 *   op 1: y = L x = d o x - Gamma_full x   (d = Gamma_full 1; the diagonal
 *                                           cancels, Sec. 2.3)
 *   op 2: y = (alpha I + L) x
 * precision: NLH_FP64, NLH_FP32 or NLH_DF32 (the NFFT stages; the output is
 * FP64).
 * A matvec is five kernel launches for n_os <= 128 (spread, the x and y
 * convolution passes in one plane kernel, the z pass, interpolation, and
 * the epilogue over the pixels; a one-window plan finishes the pixels
 * inside the interpolation) and six for n_os = 256 (three separate
 * convolution passes); the per-window contributions of a pixel are summed
 * with FP64 atomics, so results may differ between calls in the last bits.
 * Errors: NLH_ERR_ARG (bad op, precision not built, NULL pointers, op 1 or
 * 2 on a window-range plan without a reduce callback).  The call does not
 * synchronise; the NFFT kernels validate the plan's work-unit, item and
 * permutation indices, skip any that are out of range and record it, and
 * the next synchronising call on a plan reports it (NLH_ERR_CUDA). */
nlh_status nlh_matvec(nlh_plan plan, int op, int precision, double alpha,
                      const double *x, double *y, void *stream);

/* Krylov methods (Sec. 4.3 and Sec. 5.3-5.4). */
enum {
    NLH_CG = 0,            /* CG in the original basis (Table 2)              */
    NLH_PCG_JACOBI = 1,    /* CG with P_a = alpha I + diag(eta)               */
    NLH_PCG_DEFLATED = 2,  /* decoupled CG with the projected P_{U,a}         */
    NLH_CG_DEFLATED = 3    /* decoupled CG without preconditioner (I_U)       */
};
/* Arithmetic of a solve. */
enum {
    NLH_SOLVE_FP64 = 0,    /* every matvec FP64                               */
    NLH_SOLVE_MIXED = 1,   /* FP32-NFFT inner solves inside iterative
                              refinement whose residuals use the FP64-accurate
                              operator (double-float if the plan has it,
                              else FP64); dots always FP64                    */
    NLH_SOLVE_DF32 = 2     /* every matvec double-float                       */
};

typedef struct {
    double tol;             /* stop at ||b - A u|| <= tol ||b||               */
    int maxit;              /* CG iterations (per inner solve when mixed)     */
    int method;             /* NLH_CG .. NLH_CG_DEFLATED                      */
    int arith;              /* NLH_SOLVE_FP64 or NLH_SOLVE_MIXED              */
    double inner_tol;       /* mixed: inner relative tolerance of a refinement
                               step.  > 0: fixed; a step that can end the solve
                               (tol / (2 rel) >= max(inner_tol / 4, 1e-4), rel
                               the current relative residual) runs to
                               min(tol / (2 rel), 0.1) instead.  <= 0
                               (automatic): every step runs to tol / rel
                               clamped to [1e-7, 0.1], so the first step aims
                               at tol and one FP64-accurate residual often
                               ends the solve; an inner solve also ends when
                               its best residual has not fallen by 30 % for 3
                               iterations within 8x of its target, or for 9
                               anywhere (the FP32 operator's rounding floor) */
    int max_outer;          /* mixed: refinement steps (0 = 20)               */
    const double *x0;       /* device N, initial guess, or NULL (zero)        */
    const double *diag_scale; /* device N, positive factors c_i multiplying
                               P_a (learned correction), or NULL             */
    double *hist;           /* HOST, optional residual history ||r_k||/||b||  */
    int hist_len;           /* capacity of hist                               */
    int check_every;        /* 0: the whole Krylov loop runs on the device as
                               one CUDA graph with a WHILE conditional node
                               (no host round trip); k > 0: host-driven loop
                               checking convergence every k iterations       */
    int x0_check;           /* 1: use x0 only if its residual is below that of
                               the method's own start ((mean(b)/alpha) 1 for
                               the deflated methods, 0 otherwise), else start
                               there (info.x0_rejected); 0: use x0 as given */
    int precond;            /* preconditioner of NLH_PCG_JACOBI and
                               NLH_PCG_DEFLATED: 0 P_a = alpha + max(d-1, 0)
                               (Jacobi), 1 P_b' = sqrt(P_a^2 + (d'-1)/L)
                               with d' = Gamma_full 1 at sigma/sqrt(2)
                               (Sec. 4.3.3, Eq. ANOVA_Norm_2_Prec); d' is
                               computed once per plan and sigma           */
} nlh_solve_opts;

typedef struct {
    int iters;              /* CG iterations (summed over inner solves)       */
    int outer;              /* refinement steps (1 for FP64 solves)           */
    int matvecs_fp64, matvecs_fp32;
    double rel_res;         /* last recurrence residual ||r||/||b||           */
    double rel_res_true;    /* ||b - A u||/||b|| from a final FP64 matvec     */
    double seconds;         /* wall time of the call                          */
    int used_fallback;      /* 1 if diag_scale was dropped after a failure    */
    int status;             /* same as the return value                       */
    int x0_rejected;        /* 1 if x0 was not used: its residual was not
                               below that of the method's own start          */
} nlh_solve_info;

/* Solve (alpha I + L) u = b (Eq. discretized-state with mu = 1).
 * NLH_PCG_DEFLATED: u = (mean(b)/alpha) 1 + w with w the CG iterate on the
 * orthogonal complement of 1, preconditioned by Pi P^-1 Pi (Pi the mean
 * removal); this is iterate-for-iterate the paper's CG on pi_2(U^T A U)
 * with pi_2(U^T P_a^-1 U) (Sec. 4.3.2), because U = [1/sqrt(n), U_2] and
 * U_2 U_2^T = Pi.  b, u device FP64 length N; u is overwritten.
 * Synchronises `stream`.  Returns NLH_OK, NLH_ERR_NOT_CONVERGED (u = last
 * iterate), NLH_ERR_BREAKDOWN, or an error. */
nlh_status nlh_solve(nlh_plan plan, double alpha, const double *b, double *u,
                     const nlh_solve_opts *opts, nlh_solve_info *info,
                     void *stream);

/* Many solves at once (the batched form of the bilevel sweep): solve i is
 * (alphas[i] I + L_i) u[i] = b[i] with the operator of plans[i] (each plan
 * carries its own image, sigma and NFFT parameters).  The whole batch is
 * one CUDA graph, launched once on `stream`: each solve is a branch that
 * runs its complete solve on the device (for NLH_SOLVE_MIXED the refinement
 * loop is a device-side WHILE over steps, each an inner FP32 Krylov solve
 * (itself a WHILE over CG iterations), the FP64-accurate residual and a
 * decision kernel), branches of distinct plans run concurrently and solves
 * that share a plan follow one another in one branch.  The graph is cached
 * for the sequence of plans and options (at most 4 kept); it owns staging
 * buffers for the right-hand sides and solutions (2 x the sum of N doubles),
 * so the call copies b[i] in and u[i] out around the launch.  Plans with a
 * reduce callback run round by round instead (one graph per solve and
 * refinement step, on a pool of internal streams).  opts applies to every
 * solve; x0 and diag_scale must be NULL.  b[i], u[i] are device vectors of
 * the plan's N.  Work is ordered after `stream`; the call synchronises and
 * fills infos[i] (seconds = wall time of the whole batch).  Returns the
 * worst status. */
nlh_status nlh_solve_batched(int nsolves, const nlh_plan *plans, const double *alphas,
                             const double *const *b, double *const *u,
                             const nlh_solve_opts *opts, nlh_solve_info *infos,
                             void *stream);

/* Free a plan and everything it owns.  NULL is accepted. */
nlh_status nlh_plan_destroy(nlh_plan plan);

/* Message of the last error on the calling thread ("" if none). */
const char *nlh_last_error(void);

/* Library version string. */
const char *nlh_version(void);

/* Residual norms with no device allocation.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory when they need a
 * residual -- code running while a framework captures a CUDA graph (where
 * cudaMalloc is not allowed), real-time loops that must not pay allocation
 * latency, processes whose device memory belongs to another allocator.
 *   b, q   device FP64, length N (typically q = (alpha I + L) u from
 *          nlh_matvec, op 2)
 *   res    device FP64, length N, receives b - q; may be NULL
 *   norms  device FP64, 2 values: ||b - q||_2 and ||b||_2
 * The per-block partial sums go to one fixed array inside the library
 * (128 KiB, allocated when the library is loaded on each device and kept
 * until the process exits), so N is limited to 33,554,432 (8192 blocks of
 * 4096 elements); larger N returns NLH_ERR_ARG.  Nothing in the array must
 * start at zero: every call overwrites the slots it reads.  All calls, on
 * every stream, share that array, so calls that overlap on the GPU race and
 * must be ordered by the caller.  A call outside stream capture looks up
 * the array's device address (cudaGetSymbolAddress, with the calling
 * thread's current device); a call on a stream that is being captured uses
 * the address of the last call outside capture on that device, so make one
 * call on each device before any capture (after a device reset, again).
 * The call allocates nothing and does not synchronise. */
nlh_status nlh_residual_norms_noalloc(const double *b, const double *q,
                                      int64_t N, double *res, double *norms,
                                      void *stream);

/* ---- Instrumentation (not part of the paper's method) ------------------
 * nlh_kernel_launches: number of CUDA kernels the library has launched in
 * this process.  nlh_profile_enable(1) makes the library bracket each launch
 * of the classes below with CUDA events on the launch's own stream;
 * nlh_profile_read synchronises those events and returns the launch count
 * and summed device time of one class; nlh_profile_reset drops the records.
 * Profiling is process-wide and off by default. */
enum {
    NLH_K_SPREAD64 = 0, NLH_K_SPREAD32, NLH_K_CONV64, NLH_K_CONV32,
    NLH_K_INTERP64, NLH_K_INTERP32, NLH_K_EPILOGUE, NLH_K_KRYLOV, NLH_K_PLAN,
    NLH_K_SPREADDF, NLH_K_INTERPDF, NLH_K_NCLASSES
};
int64_t nlh_kernel_launches(void);
nlh_status nlh_profile_enable(int enable);
nlh_status nlh_profile_reset(void);
nlh_status nlh_profile_read(int kernel_class, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* NLH_H */
