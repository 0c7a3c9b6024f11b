// solve.cu -- Krylov solves of (alpha I + L) u = b on the device.
//
// Paper: arXiv 2407.06834.  CG and Jacobi-PCG in the original basis
// (Sec. 5.3, Sec. 5.4, P_a = lambda I + mu diag(eta), Sec. 4.3.1) and the
// decoupled CG with the projected preconditioner P_{U,a} (Sec. 4.1 and
// Sec. 4.3.2).  The decoupled method is run in the equivalent form
//   u = (mean(b)/alpha) 1 + w,  w on the orthogonal complement of 1,
//   CG on w with preconditioner Pi P_a^-1 Pi, Pi = I - 1 1^T / N,
// which gives the same iterates as the paper's CG on pi_2(U^T A U) with
// pi_2(U^T P_a^-1 U): U = [1/sqrt(N), U_2] (Eq. ULap) and U_2 U_2^T = Pi, so
// every CG scalar (r^T z, p^T A p) agrees.  The first block of the paper's
// change of basis, x_1 = g_1 / lambda, is the mean(b)/alpha term.
//
// Each CG iteration is one matvec (nfft.cu, with p^T A p fused into its
// epilogue) and two vector kernels.  Scalars stay on the device; a `done`
// flag makes every kernel of an iteration that was queued after convergence
// return at once, so the host checks convergence only every few iterations.
#include "common.cuh"

#include <chrono>
#include <cmath>

namespace nlh {

// Partials layout: stats at partials[b * 4 + j] (j = 0..3), the matvec
// epilogue's x^T y at partials[4 * kRedBlocks + b].
__device__ __forceinline__ double *pq_parts(double *partials) { return partials + 4 * kRedBlocks; }

// ------------------------------------------------------------------ kernels
// pinv = 1 / (c o (alpha + max(d - 1, 0))) for Jacobi (eta = d - 1, the
// exact diagonal 1 removed), or 1.
__global__ void k_pinv(const double *__restrict__ d, const double *__restrict__ c, double alpha,
                       int precond, int64_t N, double *__restrict__ pinv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = 1.0;
        if (precond) {
            double eta = fmax(d[i] - 1.0, 0.0);
            double P = alpha + eta;
            if (c) P *= c[i];
            v = 1.0 / P;
        }
        pinv[i] = v;
    }
}

// r = rhs - q (q = A x0) or rhs; partials: sum r, sum rhs^2, sum rhs.
__global__ void __launch_bounds__(kRedThreads)
k_init1(const double *__restrict__ rhs, const double *__restrict__ q, int64_t N,
        double *__restrict__ r, double *__restrict__ partials) {
    __shared__ double sh[33];
    double s_r = 0, s_b2 = 0, s_b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double b = rhs[i];
        double ri = q ? b - q[i] : b;
        r[i] = ri;
        s_r += ri;
        s_b2 = fma(b, b, s_b2);
        s_b += b;
    }
    double v0 = block_sum(s_r, sh), v1 = block_sum(s_b2, sh), v2 = block_sum(s_b, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 4 + 0] = v0;
        partials[blockIdx.x * 4 + 1] = v1;
        partials[blockIdx.x * 4 + 2] = v2;
        partials[blockIdx.x * 4 + 3] = 0.0;
    }
}

// Deflation of r (if deflate), t = pinv o r; partials: sum t, r.t, r.r, sum r.
// Block 0 records ||rhs|| and mean(rhs).
__global__ void __launch_bounds__(kRedThreads)
k_init2(double *__restrict__ r, const double *__restrict__ pinv, int64_t N, int deflate,
        double *__restrict__ t, double *__restrict__ partials, double *__restrict__ partials2,
        SolveState *__restrict__ st) {
    __shared__ double sh[33];
    double sum_r0 = reduce_partials(partials, gridDim.x, 4, 0, sh);
    double sum_b2 = reduce_partials(partials, gridDim.x, 4, 1, sh);
    double sum_b = reduce_partials(partials, gridDim.x, 4, 2, sh);
    double rmean = deflate ? sum_r0 / (double)N : 0.0;
    double st_ = 0, srt = 0, srr = 0, sr = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double ri = r[i] - rmean;
        r[i] = ri;
        double ti = pinv[i] * ri;
        t[i] = ti;
        st_ += ti;
        srt = fma(ri, ti, srt);
        srr = fma(ri, ri, srr);
        sr += ri;
    }
    double v0 = block_sum(st_, sh), v1 = block_sum(srt, sh), v2 = block_sum(srr, sh),
           v3 = block_sum(sr, sh);
    if (threadIdx.x == 0) {
        partials2[blockIdx.x * 4 + 0] = v0;
        partials2[blockIdx.x * 4 + 1] = v1;
        partials2[blockIdx.x * 4 + 2] = v2;
        partials2[blockIdx.x * 4 + 3] = v3;
        if (blockIdx.x == 0) {
            st->bnorm = sqrt(sum_b2);
            st->bmean = sum_b / (double)N;
        }
    }
}

// Shared tail of the init and direction kernels: from the stats partials
// (sum t, r.t, r.r, sum r) form z = t - mean(t) (deflated) or t, then
// p = z + beta p.  Block 0 records the scalars and the convergence flag.
__global__ void __launch_bounds__(kRedThreads)
k_direction(const double *__restrict__ t, double *__restrict__ p, int64_t N, int deflate,
            int first, const double *__restrict__ partials, SolveState *__restrict__ st,
            double *__restrict__ hist) {
    __shared__ double sh[33];
    if (st->done) return;
    double sum_t = reduce_partials(partials, gridDim.x, 4, 0, sh);
    double rt = reduce_partials(partials, gridDim.x, 4, 1, sh);
    double rr = reduce_partials(partials, gridDim.x, 4, 2, sh);
    double sum_r = reduce_partials(partials, gridDim.x, 4, 3, sh);
    double tmean = deflate ? sum_t / (double)N : 0.0;
    double rz = rt - tmean * sum_r;  // r^T (t - tmean 1)
    double beta = first ? 0.0 : rz / st->rz_old;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double z = t[i] - tmean;
        p[i] = first ? z : fma(beta, p[i], z);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int k = first ? 0 : st->k + 1;
        double bn = st->bnorm > 0.0 ? st->bnorm : 1.0;
        double rel = sqrt(rr) / bn;
        st->k = k;
        st->rz = rz;
        st->rr = rr;
        if (k < kMaxHist) hist[k] = rel;
        if (!(rel == rel)) {               // NaN residual: breakdown
            st->status = -4;
            st->done = 1;
        } else if (rel <= st->tol || k >= st->maxit) {
            st->done = 1;
        }
    }
}

// CG update with the p^T A p partials of the matvec epilogue:
// a = r^T z / p^T A p, w += a p, r -= a q, t = pinv o r.
__global__ void __launch_bounds__(kRedThreads)
k_update(double *__restrict__ w, double *__restrict__ r, const double *__restrict__ p,
         const double *__restrict__ q, const double *__restrict__ pinv, double *__restrict__ t,
         int64_t N, double *__restrict__ partials, SolveState *__restrict__ st) {
    __shared__ double sh[33];
    if (st->done) return;
    double pq = reduce_partials(pq_parts(partials), kRedBlocks, 1, 0, sh);
    double rz = st->rz;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = -4;
            st->done = 1;
        }
        return;
    }
    double a = rz / pq;
    double st_ = 0, srt = 0, srr = 0, sr = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        w[i] = fma(a, p[i], w[i]);
        double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        double ti = pinv[i] * ri;
        t[i] = ti;
        st_ += ti;
        srt = fma(ri, ti, srt);
        srr = fma(ri, ri, srr);
        sr += ri;
    }
    double v0 = block_sum(st_, sh), v1 = block_sum(srt, sh), v2 = block_sum(srr, sh),
           v3 = block_sum(sr, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 4 + 0] = v0;
        partials[blockIdx.x * 4 + 1] = v1;
        partials[blockIdx.x * 4 + 2] = v2;
        partials[blockIdx.x * 4 + 3] = v3;
        if (blockIdx.x == 0) st->rz_old = rz;
    }
}

// w = x0 with its mean removed (deflated) or x0; w = 0 if x0 == NULL.
__global__ void k_start(const double *__restrict__ x0, int64_t N, double mean,
                        double *__restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = x0 ? x0[i] - mean : 0.0;
}

// out = (accumulate ? out : 0) + w + shift
__global__ void k_finish(const double *__restrict__ w, int64_t N, const SolveState *st,
                         double inv_alpha, int deflate, int accumulate, double *__restrict__ out) {
    double shift = deflate ? st->bmean * inv_alpha : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = w[i] + shift;
        out[i] = accumulate ? out[i] + v : v;
    }
}

// res = b - q; partials: sum res^2, sum b^2.
__global__ void __launch_bounds__(kRedThreads)
k_residual(const double *__restrict__ b, const double *__restrict__ q, int64_t N,
           double *__restrict__ res, double *__restrict__ partials) {
    __shared__ double sh[33];
    double s_rr = 0, s_bb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double bi = b[i], ri = bi - q[i];
        if (res) res[i] = ri;
        s_rr = fma(ri, ri, s_rr);
        s_bb = fma(bi, bi, s_bb);
    }
    double v0 = block_sum(s_rr, sh), v1 = block_sum(s_bb, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 2 + 0] = v0;
        partials[blockIdx.x * 2 + 1] = v1;
    }
}

// ------------------------------------------------------------------ host drivers
struct KrylovResult {
    int iters = 0;
    int status = 0;  // 0 ok, 1 not converged, -4 breakdown
    double rel = 0;  // last recurrence residual relative to ||rhs||
    int matvecs = 0;
};

static double *pq_parts_host(Plan &P) { return P.partials + 4 * kRedBlocks; }

static double host_sum_partials(Plan &P, int count, int stride, int off, cudaStream_t s) {
    std::vector<double> h((size_t)count * stride);
    NLH_CUDA(cudaMemcpyAsync(h.data(), P.partials, sizeof(double) * count * stride,
                             cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    double v = 0.0;
    for (int j = 0; j < count; ++j) v += h[(size_t)j * stride + off];
    return v;
}

// One Krylov solve A x = rhs with the NFFT matvec of precision `prec`.
// x_out = solution (overwritten, or accumulated into if `accumulate`).
static KrylovResult krylov(Plan &P, int prec, double alpha, const double *rhs, const double *x0,
                           double *x_out, int accumulate, double tol, int maxit, int method,
                           const double *diag_scale, int check_every, cudaStream_t s) {
    const int64_t N = P.N;
    const int deflate = (method == NLH_PCG_DEFLATED || method == NLH_CG_DEFLATED);
    const int precond = (method == NLH_PCG_JACOBI || method == NLH_PCG_DEFLATED);
    const double *d = P.d64 ? P.d64 : (P.ddf ? P.ddf : P.d32);
    KrylovResult res;
    const int B = kRedBlocks, T = kRedThreads;
    double *part2 = P.partials + 5 * kRedBlocks;  // second stats region (init only)

    SolveState init{};
    init.tol = tol;
    init.maxit = maxit;
    init.rz_old = 1.0;
    NLH_CUDA(cudaMemcpyAsync(P.st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    k_pinv<<<B, T, 0, s>>>(d, diag_scale, alpha, precond, N, P.pinv);
    NLH_CHECK_LAUNCH();
    // start vector and initial residual
    const double *qptr = nullptr;
    if (x0) {
        double mean = 0.0;
        if (deflate) {
            k_init1<<<B, T, 0, s>>>(x0, nullptr, N, P.t, P.partials);  // sum x0 in slot 0
            NLH_CHECK_LAUNCH();
            mean = host_sum_partials(P, B, 4, 0, s) / (double)N;
        }
        k_start<<<B, T, 0, s>>>(x0, N, mean, P.w);
        NLH_CHECK_LAUNCH();
        matvec(P, 2, prec, alpha, P.w, P.q, nullptr, nullptr, s);
        res.matvecs++;
        qptr = P.q;
    } else {
        k_start<<<B, T, 0, s>>>(nullptr, N, 0.0, P.w);
        NLH_CHECK_LAUNCH();
    }
    k_init1<<<B, T, 0, s>>>(rhs, qptr, N, P.r, P.partials);
    NLH_CHECK_LAUNCH();
    k_init2<<<B, T, 0, s>>>(P.r, P.pinv, N, deflate, P.t, P.partials, part2, P.st);
    NLH_CHECK_LAUNCH();
    k_direction<<<B, T, 0, s>>>(P.t, P.p, N, deflate, 1, part2, P.st, P.hist);
    NLH_CHECK_LAUNCH();

    const int ce = check_every > 0 ? check_every : 4;
    int launched = 0;
    while (true) {
        for (int j = 0; j < ce && launched < maxit; ++j, ++launched) {
            matvec(P, 2, prec, alpha, P.p, P.q, pq_parts_host(P), &P.st->done, s);
            k_update<<<B, T, 0, s>>>(P.w, P.r, P.p, P.q, P.pinv, P.t, N, P.partials, P.st);
            NLH_CHECK_LAUNCH();
            k_direction<<<B, T, 0, s>>>(P.t, P.p, N, deflate, 0, P.partials, P.st, P.hist);
            NLH_CHECK_LAUNCH();
        }
        NLH_CUDA(cudaMemcpyAsync(P.st_host, P.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        NLH_CUDA(cudaStreamSynchronize(s));
        if (P.st_host->done || launched >= maxit) break;
    }
    const SolveState &h = *P.st_host;
    res.iters = h.k;
    res.matvecs += h.k;
    res.rel = std::sqrt(h.rr) / (h.bnorm > 0 ? h.bnorm : 1.0);
    if (h.status == -4)
        res.status = -4;
    else
        res.status = (res.rel <= tol) ? 0 : 1;
    k_finish<<<B, T, 0, s>>>(P.w, N, P.st, 1.0 / alpha, deflate, accumulate, x_out);
    NLH_CHECK_LAUNCH();
    return res;
}

// ||b - A u|| / ||b|| with the matvec arithmetic `prec`; res (optional)
// receives b - A u.
static double true_residual(Plan &P, int prec, double alpha, const double *b, const double *u,
                            double *res, cudaStream_t s) {
    matvec(P, 2, prec, alpha, u, P.q, nullptr, nullptr, s);
    k_residual<<<kRedBlocks, kRedThreads, 0, s>>>(b, P.q, P.N, res, P.partials);
    NLH_CHECK_LAUNCH();
    std::vector<double> h(2 * kRedBlocks);
    NLH_CUDA(cudaMemcpyAsync(h.data(), P.partials, sizeof(double) * 2 * kRedBlocks,
                             cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    double rr = 0, bb = 0;
    for (int j = 0; j < kRedBlocks; ++j) {
        rr += h[2 * j];
        bb += h[2 * j + 1];
    }
    return std::sqrt(rr) / (bb > 0 ? std::sqrt(bb) : 1.0);
}

}  // namespace nlh

using namespace nlh;

extern "C" nlh_status nlh_solve(nlh_plan plan, double alpha, const double *b, double *u,
                                const nlh_solve_opts *opts, nlh_solve_info *info,
                                void *stream) {
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    nlh_solve_info inf{};
    nlh_status ret = NLH_OK;
    try {
        NLH_REQUIRE(plan && b && u && opts, "nlh_solve: NULL pointer");
        NLH_REQUIRE(b != u, "nlh_solve: b and u must not alias");
        NLH_REQUIRE(alpha > 0.0 && std::isfinite(alpha), "nlh_solve: alpha=%g must be > 0", alpha);
        NLH_REQUIRE(opts->tol > 0.0 && opts->maxit >= 1 && opts->maxit < kMaxHist,
                    "nlh_solve: tol=%g maxit=%d", opts->tol, opts->maxit);
        NLH_REQUIRE(opts->method >= NLH_CG && opts->method <= NLH_CG_DEFLATED,
                    "nlh_solve: method=%d", opts->method);
        NLH_REQUIRE(opts->arith >= NLH_SOLVE_FP64 && opts->arith <= NLH_SOLVE_DF32,
                    "nlh_solve: arith=%d", opts->arith);
        Plan &P = *plan;
        cudaStream_t s = (cudaStream_t)stream;
        P.stream = s;
        // the FP64-accurate arithmetic: double-float if built, else FP64
        const int accurate = (P.precision & 4) ? NLH_DF32 : NLH_FP64;
        if (opts->arith == NLH_SOLVE_FP64)
            NLH_REQUIRE(P.precision & 1, "nlh_solve: FP64 solve needs a plan with the FP64 path");
        else if (opts->arith == NLH_SOLVE_DF32)
            NLH_REQUIRE(P.precision & 4,
                        "nlh_solve: double-float solve needs a plan with that path");
        else
            NLH_REQUIRE((P.precision & 2) && (P.precision & 5),
                        "nlh_solve: mixed solve needs the FP32 path and an FP64-accurate path");
        const int solve_prec = opts->arith == NLH_SOLVE_FP64 ? NLH_FP64 : NLH_DF32;
        const double *scale = opts->diag_scale;
        for (int attempt = 0; attempt < 2; ++attempt) {
            const double *x0 = attempt == 0 ? opts->x0 : u;
            int ce = opts->check_every;
            int st = 0;
            inf.iters = 0;
            if (opts->arith != NLH_SOLVE_MIXED) {
                KrylovResult kr = krylov(P, solve_prec, alpha, b, x0, u, 0, opts->tol,
                                         opts->maxit, opts->method, scale, ce, s);
                inf.iters = kr.iters;
                inf.outer = 1;
                inf.matvecs_fp64 += kr.matvecs + 1;
                inf.rel_res = kr.rel;
                if (opts->hist && opts->hist_len > 0) {
                    int cnt = std::min(opts->hist_len, kr.iters + 1);
                    NLH_CUDA(cudaMemcpyAsync(opts->hist, P.hist, sizeof(double) * cnt,
                                             cudaMemcpyDeviceToHost, s));
                }
                inf.rel_res_true = true_residual(P, solve_prec, alpha, b, u, nullptr, s);
                st = kr.status;
            } else {
                const double inner = opts->inner_tol > 0 ? opts->inner_tol : 1e-4;
                const int max_outer = opts->max_outer > 0 ? opts->max_outer : 20;
                double rel;
                if (x0) {
                    if (x0 != u)
                        NLH_CUDA(cudaMemcpyAsync(u, x0, sizeof(double) * P.N,
                                                 cudaMemcpyDeviceToDevice, s));
                    rel = true_residual(P, accurate, alpha, b, u, P.rhs, s);
                    inf.matvecs_fp64 += 1;
                } else {
                    NLH_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * P.N, s));
                    NLH_CUDA(cudaMemcpyAsync(P.rhs, b, sizeof(double) * P.N,
                                             cudaMemcpyDeviceToDevice, s));
                    rel = 1.0;
                }
                int outer = 0;
                st = 1;
                while (rel > opts->tol && outer < max_outer) {
                    KrylovResult kr = krylov(P, NLH_FP32, alpha, P.rhs, nullptr, u, 1, inner,
                                             opts->maxit, opts->method, scale, ce, s);
                    inf.iters += kr.iters;
                    inf.matvecs_fp32 += kr.matvecs;
                    ++outer;
                    if (kr.status == -4) { st = -4; break; }
                    rel = true_residual(P, accurate, alpha, b, u, P.rhs, s);
                    inf.matvecs_fp64 += 1;
                    if (opts->hist && outer - 1 < opts->hist_len) opts->hist[outer - 1] = rel;
                }
                if (st != -4) st = rel <= opts->tol ? 0 : 1;
                inf.outer = outer;
                inf.rel_res = rel;
                inf.rel_res_true = rel;
            }
            if (st == 0 || !scale || attempt == 1) {
                ret = st == 0 ? NLH_OK : (st == -4 ? NLH_ERR_BREAKDOWN : NLH_ERR_NOT_CONVERGED);
                break;
            }
            // the learned correction failed: restart plain from the last iterate
            scale = nullptr;
            inf.used_fallback = 1;
        }
        check_device_error(P, s);
    } catch (Failure &f) {
        ret = f.st;
    }
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inf.status = ret;
    if (info) *info = inf;
    return ret;
}
