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
#include <map>
#include <memory>
#include <mutex>

namespace nlh {

// Partials layout: stats at partials[b * 4 + j] (j = 0..3), the second set
// of the start-up at partials[5 * kRedBlocks + b * 4 + j], the matvec
// epilogue's x^T y at partials[12 * kRedBlocks + b] (kPqSlots blocks).
__device__ __forceinline__ double *pq_parts(double *partials) { return partials + 12 * kRedBlocks; }

// ------------------------------------------------------------------ kernels
// pinv = 1 / (c o P) with P the Jacobi diagonal P_a = alpha + max(d - 1, 0)
// (eta = d - 1, the exact diagonal 1 removed), or with pb2 given the P_b'
// of Sec. 4.3.3, P = sqrt(P_a^2 + pb2) (Eq. ANOVA_Norm_2_Prec with mu = 1);
// or 1 without preconditioner.  alpha is read from the solve state.
__global__ void k_pinv(const double *__restrict__ d, const double *__restrict__ c,
                       const double *__restrict__ pb2, const SolveState *__restrict__ st,
                       int precond, int64_t N, double *__restrict__ pinv) {
    const double alpha = st->alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = 1.0;
        if (precond) {
            double eta = fmax(d[i] - 1.0, 0.0);
            double P = alpha + eta;
            if (pb2) P = sqrt(P * P + pb2[i]);
            if (c) P *= c[i];
            v = 1.0 / P;
        }
        pinv[i] = v;
    }
}

__global__ void k_ones(double *__restrict__ x, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 1.0;
}

// pb2 = max(d' - 1, 0) / L: sum_l (Gamma_l o Gamma_l) 1 (zero diagonal) over
// L^2, from d' = Gamma_full 1 at sigma / sqrt 2 (the per-window kernel
// squared is the kernel at sigma / sqrt 2, and Gamma_full averages the L
// per-window sums, each with its diagonal 1).
__global__ void k_pb2(double *__restrict__ v, int64_t N, double inv_l) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = fmax(v[i] - 1.0, 0.0) * inv_l;
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

// The stopping rule after iteration k with relative residual rel: breakdown
// on a NaN residual; done at rel <= tol or k == maxit; and, with stag > 0,
// done once the best residual so far has not fallen by 30 % for `stag`
// iterations while rel is within 8x of tol, or for 3 stag iterations
// anywhere (the operator's rounding floor: the recurrence residual stops
// falling there; the wider limit away from tol keeps a plateau of CG's
// descent from ending the solve early, yet bounds a floor far above tol).
__host__ __device__ static void convergence_step(SolveState *st, double rel, int k) {
    if (!(rel == rel)) {  // NaN residual: breakdown
        st->status = -4;
        st->done = 1;
    } else if (rel <= st->tol || k >= st->maxit) {
        st->done = 1;
    } else if (st->stag > 0) {
        if (!(st->best > 0.0) || rel < 0.7 * st->best) {
            st->best = rel;
            st->k_best = k;
        } else if (k - st->k_best >= (rel <= 8.0 * st->tol ? st->stag : 3 * st->stag)) {
            st->done = 1;
        }
    }
}

// Shared tail of the init and direction kernels: from the stats partials
// (sum t, r.t, r.r, sum r) form z = t - mean(t) (deflated) or t, then
// p = z + beta p.  Block 0 records the scalars and the convergence flag.
// cond != 0: the WHILE node of a solve graph; block 0 sets it to continue
// (1) or stop (0) on every path, so the device-side loop always ends once
// `done` is set (converged, broken down, or k == maxit).
__device__ __forceinline__ void set_loop(unsigned long long cond, const SolveState *st) {
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, st->done ? 0u : 1u);
}

__global__ void __launch_bounds__(kRedThreads)
k_direction(const double *__restrict__ t, double *__restrict__ p, int64_t N, int deflate,
            int first, const double *__restrict__ partials, SolveState *__restrict__ st,
            double *__restrict__ hist, unsigned long long cond) {
    __shared__ double sh[33];
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_loop(cond, st);
        return;
    }
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
        convergence_step(st, rel, k);
        set_loop(cond, st);
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
    double pq = reduce_partials(pq_parts(partials), kPqSlots, 1, 0, sh);
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

// w = x0 with its mean removed (deflated; the sum of x0 is in partials
// slot 0 of the previous k_init1) or x0; w = 0 if x0 == NULL.
__global__ void __launch_bounds__(kRedThreads)
k_start(const double *__restrict__ x0, int64_t N, const double *__restrict__ partials,
        int deflate, double *__restrict__ w) {
    __shared__ double sh[33];
    double mean = 0.0;
    if (x0 && deflate) mean = reduce_partials(partials, gridDim.x, 4, 0, sh) / (double)N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = x0 ? x0[i] - mean : 0.0;
}

// out = (accumulate ? out : 0) + w + shift, shift = mean(rhs)/alpha for the
// deflated methods (the exactly solved first block).
__global__ void k_finish(const double *__restrict__ w, int64_t N, const SolveState *st,
                         int deflate, int accumulate, double *__restrict__ out) {
    double shift = deflate ? st->bmean / st->alpha : 0.0;
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
    double s_rr = 0, s_bb = 0, s_b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double bi = b[i], ri = bi - q[i];
        if (res) res[i] = ri;
        s_rr = fma(ri, ri, s_rr);
        s_bb = fma(bi, bi, s_bb);
        s_b += bi;
    }
    double v0 = block_sum(s_rr, sh), v1 = block_sum(s_bb, sh), v2 = block_sum(s_b, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 3 + 0] = v0;
        partials[blockIdx.x * 3 + 1] = v1;
        partials[blockIdx.x * 3 + 2] = v2;
    }
}

// ------------------------------------------------------------------ host drivers
// The P_b' term of the plan for its current sigma (computed once per sigma):
// a degree matvec with the multiplier tables of sigma / sqrt 2 (the torus
// map and the window weights do not depend on sigma), in the plan's most
// accurate arithmetic.
void ensure_pb2(Plan &P, cudaStream_t s) {
    if (P.pb2 && P.pb2_sigma == P.sigma) return;
    if (!P.pb2) P.pb2 = P.alloc<double>(P.N);
    const double sig = P.sigma;
    P.sigma = sig / std::sqrt(2.0);
    try {
        plan_tables(P, s);
        k_ones<<<kRedBlocks, kRedThreads, 0, s>>>(P.t, P.N);
        NLH_CHECK_LAUNCH();
        const int prec = (P.precision & 1) ? NLH_FP64 : (P.precision & 4) ? NLH_DF32 : NLH_FP32;
        matvec(P, 0, prec, 0.0, P.t, P.pb2, nullptr, nullptr, s);
        k_pb2<<<kRedBlocks, kRedThreads, 0, s>>>(P.pb2, P.N, 1.0 / P.L);
        NLH_CHECK_LAUNCH();
    } catch (...) {
        P.sigma = sig;
        plan_tables(P, s);
        throw;
    }
    P.sigma = sig;
    plan_tables(P, s);
    P.pb2_sigma = sig;
}

struct KrylovResult {
    int iters = 0;
    int status = 0;  // 0 ok, 1 not converged, -4 breakdown
    double rel = 0;  // last recurrence residual relative to ||rhs||
    int matvecs = 0;
};

static double *pq_parts_host(Plan &P) { return P.partials + 12 * kRedBlocks; }

static void method_flags(int method, int &deflate, int &precond) {
    deflate = (method == NLH_PCG_DEFLATED || method == NLH_CG_DEFLATED);
    precond = (method == NLH_PCG_JACOBI || method == NLH_PCG_DEFLATED);
}

// Start of a solve: preconditioner, start vector, initial residual and first
// direction.  The right-hand side is P.rhs, the warm start P.x0, the
// optional diagonal scale P.cbuf; alpha, tol, maxit come from P.st.
static void enqueue_init(Plan &P, int prec, int method, bool has_x0, bool has_scale,
                         unsigned long long cond, cudaStream_t s) {
    int deflate, precond;
    method_flags(method, deflate, precond);
    const int64_t N = P.N;
    const int B = kRedBlocks, T = kRedThreads;
    const double *d = P.d64 ? P.d64 : (P.ddf ? P.ddf : P.d32);
    double *part2 = P.partials + 5 * kRedBlocks;
    k_pinv<<<B, T, 0, s>>>(d, has_scale ? P.cbuf : nullptr, P.pc_kind == 1 ? P.pb2 : nullptr,
                           P.st, precond, N, P.pinv);
    NLH_CHECK_LAUNCH();
    const double *qptr = nullptr;
    if (has_x0) {
        k_init1<<<B, T, 0, s>>>(P.x0, nullptr, N, P.t, P.partials);  // sum x0 -> slot 0
        NLH_CHECK_LAUNCH();
        k_start<<<B, T, 0, s>>>(P.x0, N, P.partials, deflate, P.w);
        NLH_CHECK_LAUNCH();
        matvec(P, 2, prec, 0.0, P.w, P.q, nullptr, nullptr, s, &P.st->alpha);
        qptr = P.q;
    } else {
        k_start<<<B, T, 0, s>>>(nullptr, N, nullptr, 0, P.w);
        NLH_CHECK_LAUNCH();
    }
    k_init1<<<B, T, 0, s>>>(P.rhs, qptr, N, P.r, P.partials);
    NLH_CHECK_LAUNCH();
    k_init2<<<B, T, 0, s>>>(P.r, P.pinv, N, deflate, P.t, P.partials, part2, P.st);
    NLH_CHECK_LAUNCH();
    k_direction<<<B, T, 0, s>>>(P.t, P.p, N, deflate, 1, part2, P.st, P.hist, cond);
    NLH_CHECK_LAUNCH();
}

// One CG iteration: matvec with the fused p^T A p, update, new direction.
static void enqueue_iteration(Plan &P, int prec, int method, unsigned long long cond,
                              cudaStream_t s) {
    int deflate, precond;
    method_flags(method, deflate, precond);
    const int B = kRedBlocks, T = kRedThreads;
    matvec(P, 2, prec, 0.0, P.p, P.q, pq_parts_host(P), &P.st->done, s, &P.st->alpha);
    k_update<<<B, T, 0, s>>>(P.w, P.r, P.p, P.q, P.pinv, P.t, P.N, P.partials, P.st);
    NLH_CHECK_LAUNCH();
    k_direction<<<B, T, 0, s>>>(P.t, P.p, P.N, deflate, 0, P.partials, P.st, P.hist, cond);
    NLH_CHECK_LAUNCH();
}

// A whole solve as one CUDA graph: the start-up kernels, then a WHILE
// conditional node whose body is one iteration; the direction kernel sets
// the loop condition from the device-side convergence flag, so the solve
// runs without any host round trip.  Graphs are cached per plan.
static cudaGraphExec_t solve_graph(Plan &P, int prec, int method, bool has_x0, bool has_scale) {
    const int key = prec | (method << 2) | ((int)has_x0 << 4) | ((int)has_scale << 5) |
                    (P.pc_kind << 6);
    auto it = P.graphs.find(key);
    if (it != P.graphs.end()) return it->second;
    if (!P.capture_stream) P.capture_stream = take_capture_stream(P.device);
    cudaStream_t cs = P.capture_stream;
    cudaGraph_t top = nullptr;
    cudaGraphExec_t exec = nullptr;
    NLH_CUDA(cudaGraphCreate(&top, 0));
    try {
        cudaGraphConditionalHandle h;
        NLH_CUDA(cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault));
        NLH_CUDA(cudaStreamBeginCaptureToGraph(cs, top, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_init(P, prec, method, has_x0, has_scale, (unsigned long long)h, cs);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
            throw;
        }
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        NLH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
        std::vector<cudaGraphNode_t> leaves(deps, deps + ndeps);
        NLH_CUDA(cudaStreamEndCapture(cs, &top));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        NLH_CUDA(cudaGraphAddNode(&wnode, top, leaves.data(), nullptr, leaves.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        NLH_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_iteration(P, prec, method, (unsigned long long)h, cs);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
            throw;
        }
        NLH_CUDA(cudaStreamEndCapture(cs, &body));
        NLH_CUDA(cudaGraphInstantiate(&exec, top, 0));
    } catch (...) {
        cudaGraphDestroy(top);
        throw;
    }
    cudaGraphDestroy(top);
    P.graphs[key] = exec;
    return exec;
}

// Enqueue one Krylov solve A x = rhs (NFFT arithmetic `prec`): state and
// inputs into the plan's buffers, the solve (graph, or a host-driven loop
// when check_every > 0), x_out = solution (or += when accumulate), and a
// copy of the device state to the pinned mirror.  krylov_collect reads it
// after the stream has been synchronised.
// Relative tolerance of the inner FP32 solve of one refinement step, from
// the current FP64-accurate relative residual rel.
// - inner > 0 (the caller's fixed inner tolerance): a step whose remaining
//   reduction is within reach (tol / (2 rel) >= max(inner / 4, 1e-4)) runs
//   to exactly tol / (2 rel), capped at 0.1, so that it is the last step;
//   any other step runs to inner.
// - inner <= 0 (automatic): every step runs to tol / rel, clamped to
//   [kInnerFloor, 0.1], with the stagnation exit of kInnerStag iterations.
//   The first step from u = 0 therefore aims at the outer tolerance: where
//   the FP32 operator's rounding floor lies below it, one FP64-accurate
//   residual certifies the solve and a whole refinement step with its
//   FP64-accurate matvec is saved; where it does not, the inner CG stops at
//   the floor (stagnation exit) and a short second step follows.  The floor
//   depends on the plan (measured 6e-7 to 3e-6 relative at 512^2 and
//   2048^2), so a fixed target below it would spin to maxit.
static constexpr double kInnerFloor = 1e-7;
static constexpr int kInnerStag = 3;
__host__ __device__ static double inner_tolerance(double inner, double tol, double rel) {
    if (inner <= 0) return fmin(fmax(tol / rel, kInnerFloor), 0.1);
    const double need = 0.5 * tol / rel;
    if (need >= fmax(0.25 * inner, 1e-4)) return fmin(need, 0.1);
    return inner;
}

static void krylov_launch(Plan &P, int prec, double alpha, const double *rhs, const double *x0,
                          double *x_out, int accumulate, double tol, int maxit, int method,
                          const double *scale, int check_every, cudaStream_t s,
                          int stag = 0) {
    int deflate, precond;
    method_flags(method, deflate, precond);
    // a plan whose matvecs call a reduce callback (a window range summed over
    // ranks) runs the host-driven loop: the callback enqueues its collective
    // when the matvec is issued, which a captured graph would not repeat
    if (P.reduce_fn && check_every <= 0) check_every = 4;
    SolveState init{};
    init.tol = tol;
    init.maxit = maxit;
    init.rz_old = 1.0;
    init.alpha = alpha;
    init.stag = stag;
    *P.st_host = init;
    NLH_CUDA(cudaMemcpyAsync(P.st, P.st_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    if (rhs != P.rhs)
        NLH_CUDA(cudaMemcpyAsync(P.rhs, rhs, sizeof(double) * P.N, cudaMemcpyDeviceToDevice, s));
    if (x0) NLH_CUDA(cudaMemcpyAsync(P.x0, x0, sizeof(double) * P.N, cudaMemcpyDeviceToDevice, s));
    if (scale)
        NLH_CUDA(cudaMemcpyAsync(P.cbuf, scale, sizeof(double) * P.N, cudaMemcpyDeviceToDevice, s));
    if (check_every <= 0) {
        cudaGraphExec_t g = solve_graph(P, prec, method, x0 != nullptr, scale != nullptr);
        NLH_CUDA(cudaGraphLaunch(g, s));
        count_launch();
    } else {
        enqueue_init(P, prec, method, x0 != nullptr, scale != nullptr, 0ull, s);
        int launched = 0;
        while (true) {
            for (int j = 0; j < check_every && launched < maxit; ++j, ++launched)
                enqueue_iteration(P, prec, method, 0ull, s);
            NLH_CUDA(cudaMemcpyAsync(P.st_host, P.st, sizeof(SolveState), cudaMemcpyDeviceToHost,
                                     s));
            NLH_CUDA(cudaStreamSynchronize(s));
            if (P.st_host->done || launched >= maxit) break;
        }
    }
    k_finish<<<kRedBlocks, kRedThreads, 0, s>>>(P.w, P.N, P.st, deflate, accumulate, x_out);
    NLH_CHECK_LAUNCH();
    NLH_CUDA(cudaMemcpyAsync(P.st_host, P.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
}

static KrylovResult krylov_collect(Plan &P, int tol_ok_status_tol_dummy = 0) {
    (void)tol_ok_status_tol_dummy;
    const SolveState &h = *P.st_host;
    KrylovResult res;
    res.iters = h.k;
    res.matvecs = h.k;
    res.rel = std::sqrt(h.rr) / (h.bnorm > 0 ? h.bnorm : 1.0);
    if (h.status == -4)
        res.status = -4;
    else
        res.status = (res.rel <= h.tol) ? 0 : 1;
    return res;
}

// b - A u into res (optional) and the partial sums of ||b - A u||^2, ||b||^2
// copied to the pinned mirror; residual_collect sums them after a sync.
static void residual_launch(Plan &P, int prec, double alpha, const double *b, const double *u,
                            double *res, cudaStream_t s) {
    matvec(P, 2, prec, alpha, u, P.q, nullptr, nullptr, s);
    k_residual<<<kRedBlocks, kRedThreads, 0, s>>>(b, P.q, P.N, res, P.partials);
    NLH_CHECK_LAUNCH();
    NLH_CUDA(cudaMemcpyAsync(P.red_host, P.partials, sizeof(double) * 3 * kRedBlocks,
                             cudaMemcpyDeviceToHost, s));
}

// ||b - A u|| / ||b||; optionally also ||b - mean(b) 1|| / ||b||, the
// residual of the deflated methods' own start (mean(b) / alpha) 1 (L 1 = 0).
static double residual_collect(Plan &P, double *rel_mean_start = nullptr) {
    double rr = 0, bb = 0, bs = 0;
    for (int j = 0; j < kRedBlocks; ++j) {
        rr += P.red_host[3 * j];
        bb += P.red_host[3 * j + 1];
        bs += P.red_host[3 * j + 2];
    }
    const double nb = bb > 0 ? std::sqrt(bb) : 1.0;
    if (rel_mean_start) *rel_mean_start = std::sqrt(std::max(0.0, bb - bs * bs / P.N)) / nb;
    return std::sqrt(rr) / nb;
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
        NLH_REQUIRE(opts->precond == 0 || opts->precond == 1, "nlh_solve: precond=%d",
                    opts->precond);
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
        P.pc_kind = opts->precond;
        if (P.pc_kind == 1) ensure_pb2(P, s);
        // With x0_check a warm start is used only if its residual is below
        // that of the method's own start: (mean(b) / alpha) 1 for the
        // deflated methods, 0 for CG and Jacobi-PCG.
        const bool mixed = opts->arith == NLH_SOLVE_MIXED;
        const double *x0_user = opts->x0;
        double rel_x0 = 1.0;
        const bool screen = x0_user && opts->x0_check;
        if (screen) {
            // mixed: the residual is kept in P.rhs as the first right-hand side
            residual_launch(P, mixed ? accurate : solve_prec, alpha, b, x0_user,
                            mixed ? P.rhs : nullptr, s);
            NLH_CUDA(cudaStreamSynchronize(s));
            double rel_plain = 1.0;
            rel_x0 = residual_collect(P, &rel_plain);
            inf.matvecs_fp64 += 1;
            const bool deflated = opts->method == NLH_PCG_DEFLATED || opts->method == NLH_CG_DEFLATED;
            if (!(rel_x0 < (deflated ? rel_plain : 1.0))) {
                x0_user = nullptr;
                inf.x0_rejected = 1;
            }
        }
        for (int attempt = 0; attempt < 2; ++attempt) {
            const double *x0 = attempt == 0 ? x0_user : u;
            int ce = opts->check_every;
            int st = 0;
            inf.iters = 0;
            if (opts->arith != NLH_SOLVE_MIXED) {
                krylov_launch(P, solve_prec, alpha, b, x0, u, 0, opts->tol, opts->maxit,
                              opts->method, scale, ce, s);
                residual_launch(P, solve_prec, alpha, b, u, nullptr, s);
                NLH_CUDA(cudaStreamSynchronize(s));
                KrylovResult kr = krylov_collect(P);
                inf.iters = kr.iters;
                inf.outer = 1;
                inf.matvecs_fp64 += kr.matvecs + 1 + (x0 && attempt > 0 ? 1 : 0);
                inf.rel_res = kr.rel;
                if (opts->hist && opts->hist_len > 0) {
                    int cnt = std::min(opts->hist_len, kr.iters + 1);
                    NLH_CUDA(cudaMemcpy(opts->hist, P.hist, sizeof(double) * cnt,
                                        cudaMemcpyDeviceToHost));
                }
                inf.rel_res_true = residual_collect(P);
                st = kr.status;
            } else {
                const double inner = opts->inner_tol;  // <= 0: automatic
                const int max_outer = opts->max_outer > 0 ? opts->max_outer : 20;
                double rel;
                if (x0 && attempt == 0 && screen) {
                    // screened above: P.rhs = b - A x0
                    if (x0 != u)
                        NLH_CUDA(cudaMemcpyAsync(u, x0, sizeof(double) * P.N,
                                                 cudaMemcpyDeviceToDevice, s));
                    rel = rel_x0;
                } else if (x0) {
                    if (x0 != u)
                        NLH_CUDA(cudaMemcpyAsync(u, x0, sizeof(double) * P.N,
                                                 cudaMemcpyDeviceToDevice, s));
                    residual_launch(P, accurate, alpha, b, u, P.rhs, s);
                    NLH_CUDA(cudaStreamSynchronize(s));
                    rel = residual_collect(P);
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
                    krylov_launch(P, NLH_FP32, alpha, P.rhs, nullptr, u, 1,
                                  inner_tolerance(inner, opts->tol, rel), opts->maxit,
                                  opts->method, scale, ce, s, inner <= 0 ? kInnerStag : 0);
                    residual_launch(P, accurate, alpha, b, u, P.rhs, s);
                    NLH_CUDA(cudaStreamSynchronize(s));
                    KrylovResult kr = krylov_collect(P);
                    inf.iters += kr.iters;
                    inf.matvecs_fp32 += kr.matvecs;
                    ++outer;
                    if (kr.status == -4) { st = -4; break; }
                    rel = residual_collect(P);
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

// ------------------------------------------------------------------ batched solves
namespace nlh {

// Library-wide pool of non-blocking streams for batched solves.
static std::mutex g_pool_mu;
static std::vector<cudaStream_t> g_pool;
static std::vector<cudaEvent_t> g_pool_ev;

static void pool_reserve(int n) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    while ((int)g_pool.size() < n) {
        cudaStream_t st;
        cudaEvent_t ev;
        NLH_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        NLH_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        g_pool.push_back(st);
        g_pool_ev.push_back(ev);
    }
}

// ---------------------------------------------------------- a batch as one graph
// Every solve of a batch is one branch of a single CUDA graph, launched
// once per call: the branch stages its right-hand side, then runs the whole
// mixed-precision refinement on the device, a WHILE node over refinement
// steps whose body is the inner FP32 Krylov solve (itself a WHILE node over
// CG iterations), the accumulation of the correction, the FP64-accurate
// residual b - A u and a decision kernel that records the step and sets the
// outer loop's condition.  Solves that share a plan are chained one after
// another in the same branch (a plan's workspace serves one solve at a
// time).  The per-solve parameters (alpha, tolerances) live in device
// memory uploaded before each launch, the right-hand sides and solutions in
// buffers the graph owns, so a cached graph serves any call on the same
// plans.

// Parameters of one solve of a batch graph (device; uploaded per call).
struct BatchParams {
    double alpha, tol, inner;
    int maxit, max_outer, mixed, pad;
};
// Result of one solve of a batch graph (device; read back per call).
struct OuterState {
    int outer, status, iters, mv32, mv64, pad;
    double rel, rel_krylov;
};

__global__ void k_batch_start(OuterState *os) {
    OuterState o{};
    o.status = 1;
    o.rel = 1.0;
    o.rel_krylov = 1.0;
    *os = o;
}

// The Krylov state of the next inner solve: the tolerance of the refinement
// step from the current FP64-accurate residual (mixed), or the caller's.
__global__ void k_batch_state(const BatchParams *bp, const OuterState *os, SolveState *st) {
    SolveState v{};
    v.tol = bp->mixed ? inner_tolerance(bp->inner, bp->tol, os->rel) : bp->tol;
    v.maxit = bp->maxit;
    v.rz_old = 1.0;
    v.alpha = bp->alpha;
    v.stag = bp->mixed && bp->inner <= 0 ? kInnerStag : 0;
    *st = v;
}

// After an inner solve and the residual's partial sums (k_residual): record
// the step; the outer WHILE continues unless the solve converged, broke
// down or ran out of refinement steps.
__global__ void __launch_bounds__(kRedThreads)
k_batch_step(const BatchParams *bp, const SolveState *st, const double *partials,
             OuterState *os, unsigned long long cond) {
    __shared__ double sh[33];
    const double rr = reduce_partials(partials, kRedBlocks, 3, 0, sh);
    const double bb = reduce_partials(partials, kRedBlocks, 3, 1, sh);
    if (threadIdx.x != 0) return;
    const double rel = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    OuterState o = *os;
    o.iters += st->k;
    o.outer += 1;
    o.rel_krylov = sqrt(st->rr) / (st->bnorm > 0.0 ? st->bnorm : 1.0);
    bool stop = true;
    if (bp->mixed) {
        o.mv32 += st->k;
        if (st->status == -4) {
            o.status = -4;
        } else {
            o.mv64 += 1;
            o.rel = rel;
            if (rel <= bp->tol) o.status = 0;
            else if (o.outer >= bp->max_outer) o.status = 1;
            else stop = false;
        }
    } else {
        o.mv64 += st->k + 1;
        o.rel = rel;
        o.status = st->status == -4 ? -4 : (o.rel_krylov <= st->tol ? 0 : 1);
    }
    *os = o;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, stop ? 0u : 1u);
}

// Captures what fn enqueues into graph g after deps; returns the new leaves.
template <typename F>
static std::vector<cudaGraphNode_t> capture_into(cudaStream_t cs, cudaGraph_t g,
                                                 const std::vector<cudaGraphNode_t> &deps,
                                                 F &&fn) {
    NLH_CUDA(cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                           deps.size(), cudaStreamCaptureModeThreadLocal));
    try {
        fn(cs);
    } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        throw;
    }
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *leaf = nullptr;
    size_t nl = 0;
    NLH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &leaf, nullptr, &nl));
    std::vector<cudaGraphNode_t> out(leaf, leaf + nl);
    cudaGraph_t g_out = g;
    NLH_CUDA(cudaStreamEndCapture(cs, &g_out));
    return out;
}

static cudaGraphNode_t add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                                 cudaGraphConditionalHandle h, cudaGraph_t *body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    NLH_CUDA(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr,
                              deps.size(), &cp));
    *body = cp.conditional.phGraph_out[0];
    return node;
}

struct BatchGraph {
    std::vector<std::pair<uint64_t, unsigned>> key;  // (plan serial, graph epoch) per solve
    int arith = 0, method = 0, precond = 0, device = 0;
    int n = 0;
    cudaGraphExec_t exec = nullptr;
    double *bbuf = nullptr, *ubuf = nullptr;  // staged right-hand sides / solutions
    std::vector<int64_t> off;
    BatchParams *bp = nullptr, *bp_host = nullptr;
    OuterState *os = nullptr, *os_host = nullptr;
    ~BatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (bbuf) cudaFree(bbuf);
        if (ubuf) cudaFree(ubuf);
        if (bp) cudaFree(bp);
        if (os) cudaFree(os);
        if (bp_host) cudaFreeHost(bp_host);
        if (os_host) cudaFreeHost(os_host);
    }
};
static std::mutex g_batch_mu;
static std::vector<std::unique_ptr<BatchGraph>> g_batch;  // most recently used last
constexpr size_t kBatchGraphsKept = 4;

// The branch of solve i: stage, then the refinement loop (mixed) or one
// Krylov solve and its residual.
static std::vector<cudaGraphNode_t> batch_branch(Plan &P, cudaStream_t cs, cudaGraph_t top,
                                                 const std::vector<cudaGraphNode_t> &deps,
                                                 const double *bi, double *ui,
                                                 const BatchParams *bp, OuterState *os,
                                                 int arith, int method) {
    int deflate, precond;
    method_flags(method, deflate, precond);
    const bool mixed = arith == NLH_SOLVE_MIXED;
    const int accurate = (P.precision & 4) ? NLH_DF32 : NLH_FP64;
    const int prec = mixed ? NLH_FP32 : (arith == NLH_SOLVE_FP64 ? NLH_FP64 : NLH_DF32);
    const int rprec = mixed ? accurate : prec;
    const int64_t N = P.N;
    auto stage = [&](cudaStream_t c) {
        if (mixed) NLH_CUDA(cudaMemsetAsync(ui, 0, sizeof(double) * N, c));
        NLH_CUDA(cudaMemcpyAsync(P.rhs, bi, sizeof(double) * N, cudaMemcpyDeviceToDevice, c));
        k_batch_start<<<1, 1, 0, c>>>(os);
        NLH_CHECK_LAUNCH();
    };
    // one inner solve + residual + decision into graph g (cond: the outer
    // loop's handle, 0 for a single step)
    auto step = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t> &d0,
                    unsigned long long cond) {
        cudaGraphConditionalHandle hi;
        NLH_CUDA(cudaGraphConditionalHandleCreate(&hi, g, 1, cudaGraphCondAssignDefault));
        auto lv = capture_into(cs, g, d0, [&](cudaStream_t c) {
            k_batch_state<<<1, 1, 0, c>>>(bp, os, P.st);
            NLH_CHECK_LAUNCH();
            enqueue_init(P, prec, method, false, false, (unsigned long long)hi, c);
        });
        cudaGraph_t body;
        cudaGraphNode_t w = add_while(g, lv, hi, &body);
        capture_into(cs, body, {}, [&](cudaStream_t c) {
            enqueue_iteration(P, prec, method, (unsigned long long)hi, c);
        });
        return capture_into(cs, g, {w}, [&](cudaStream_t c) {
            k_finish<<<kRedBlocks, kRedThreads, 0, c>>>(P.w, N, P.st, deflate, mixed ? 1 : 0, ui);
            NLH_CHECK_LAUNCH();
            matvec(P, 2, rprec, 0.0, ui, P.q, nullptr, nullptr, c, &P.st->alpha);
            k_residual<<<kRedBlocks, kRedThreads, 0, c>>>(bi, P.q, N, mixed ? P.rhs : nullptr,
                                                          P.partials);
            NLH_CHECK_LAUNCH();
            k_batch_step<<<1, kRedThreads, 0, c>>>(bp, P.st, P.partials, os, cond);
            NLH_CHECK_LAUNCH();
        });
    };
    auto lv = capture_into(cs, top, deps, stage);
    if (!mixed) return step(top, lv, 0ull);
    cudaGraphConditionalHandle ho;
    NLH_CUDA(cudaGraphConditionalHandleCreate(&ho, top, 1, cudaGraphCondAssignDefault));
    cudaGraph_t body;
    cudaGraphNode_t w = add_while(top, lv, ho, &body);
    step(body, {}, (unsigned long long)ho);
    return {w};
}

static BatchGraph &batch_graph(int n, const nlh_plan *plans, int arith, int method,
                               int precond, int device) {
    std::vector<std::pair<uint64_t, unsigned>> key(n);
    for (int i = 0; i < n; ++i) key[i] = {plans[i]->serial, plans[i]->graph_epoch};
    for (size_t k = 0; k < g_batch.size(); ++k) {
        BatchGraph &G = *g_batch[k];
        if (G.key == key && G.arith == arith && G.method == method && G.precond == precond &&
            G.device == device) {
            std::unique_ptr<BatchGraph> keep = std::move(g_batch[k]);
            g_batch.erase(g_batch.begin() + k);
            g_batch.push_back(std::move(keep));
            return *g_batch.back();
        }
    }
    std::unique_ptr<BatchGraph> G(new BatchGraph());
    G->key = key;
    G->arith = arith;
    G->method = method;
    G->precond = precond;
    G->device = device;
    G->n = n;
    G->off.resize(n + 1, 0);
    for (int i = 0; i < n; ++i) G->off[i + 1] = G->off[i] + plans[i]->N;
    NLH_CUDA(cudaMalloc(&G->bbuf, sizeof(double) * G->off[n]));
    NLH_CUDA(cudaMalloc(&G->ubuf, sizeof(double) * G->off[n]));
    NLH_CUDA(cudaMalloc(&G->bp, sizeof(BatchParams) * n));
    NLH_CUDA(cudaMalloc(&G->os, sizeof(OuterState) * n));
    NLH_CUDA(cudaMallocHost(&G->bp_host, sizeof(BatchParams) * n));
    NLH_CUDA(cudaMallocHost(&G->os_host, sizeof(OuterState) * n));
    cudaStream_t cs = take_capture_stream(device);
    cudaGraph_t top = nullptr;
    NLH_CUDA(cudaGraphCreate(&top, 0));
    try {
        std::map<nlh_plan, std::vector<cudaGraphNode_t>> tail;  // last nodes of each plan's chain
        for (int i = 0; i < n; ++i) {
            Plan &P = *plans[i];
            tail[plans[i]] = batch_branch(P, cs, top, tail[plans[i]], G->bbuf + G->off[i],
                                          G->ubuf + G->off[i], G->bp + i, G->os + i, arith,
                                          method);
        }
        NLH_CUDA(cudaGraphInstantiate(&G->exec, top, 0));
    } catch (...) {
        cudaGraphDestroy(top);
        give_capture_stream(device, cs);
        throw;
    }
    cudaGraphDestroy(top);
    give_capture_stream(device, cs);
    if (g_batch.size() >= kBatchGraphsKept) g_batch.erase(g_batch.begin());
    g_batch.push_back(std::move(G));
    return *g_batch.back();
}

// Validated batch (see nlh_solve_batched) through its graph: upload the
// parameters and right-hand sides, one launch, copy the solutions out.
static nlh_status solve_batched_graph(int n, const nlh_plan *plans, const double *alphas,
                                      const double *const *b, double *const *u,
                                      const nlh_solve_opts *opts, nlh_solve_info *infos,
                                      cudaStream_t s,
                                      std::chrono::steady_clock::time_point t0) {
    int device = 0;
    NLH_CUDA(cudaGetDevice(&device));
    for (int i = 0; i < n; ++i) {
        NLH_REQUIRE(plans[i]->device == device, "nlh_solve_batched: plan %d is on device %d", i,
                    plans[i]->device);
        NLH_REQUIRE(b[i] != u[i], "nlh_solve_batched: b and u of solve %d alias", i);
    }
    for (int i = 0; i < n; ++i) {
        Plan &P = *plans[i];
        P.stream = s;
        P.pc_kind = opts->precond;  // captured into the graph (part of its key)
        if (P.pc_kind == 1) ensure_pb2(P, s);
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    const bool mixed = opts->arith == NLH_SOLVE_MIXED;
    BatchGraph &G = batch_graph(n, plans, opts->arith, opts->method, opts->precond, device);
    for (int i = 0; i < n; ++i) {
        BatchParams &q = G.bp_host[i];
        q.alpha = alphas[i];
        q.tol = opts->tol;
        q.inner = opts->inner_tol;  // <= 0: automatic
        q.maxit = opts->maxit;
        q.max_outer = opts->max_outer > 0 ? opts->max_outer : 20;
        q.mixed = mixed ? 1 : 0;
        q.pad = 0;
    }
    NLH_CUDA(cudaMemcpyAsync(G.bp, G.bp_host, sizeof(BatchParams) * n, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < n; ++i)
        NLH_CUDA(cudaMemcpyAsync(G.bbuf + G.off[i], b[i], sizeof(double) * plans[i]->N,
                                 cudaMemcpyDeviceToDevice, s));
    NLH_CUDA(cudaGraphLaunch(G.exec, s));
    count_launch();
    for (int i = 0; i < n; ++i)
        NLH_CUDA(cudaMemcpyAsync(u[i], G.ubuf + G.off[i], sizeof(double) * plans[i]->N,
                                 cudaMemcpyDeviceToDevice, s));
    NLH_CUDA(cudaMemcpyAsync(G.os_host, G.os, sizeof(OuterState) * n, cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i) check_device_error(*plans[i], s);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    nlh_status worst = NLH_OK;
    for (int i = 0; i < n; ++i) {
        const OuterState &o = G.os_host[i];
        nlh_solve_info inf{};
        inf.iters = o.iters;
        inf.outer = o.outer;
        inf.matvecs_fp32 = o.mv32;
        inf.matvecs_fp64 = o.mv64;
        inf.rel_res = mixed ? o.rel : o.rel_krylov;
        inf.rel_res_true = o.rel;
        inf.status = o.status == 0 ? NLH_OK
                                   : (o.status == -4 ? NLH_ERR_BREAKDOWN : NLH_ERR_NOT_CONVERGED);
        inf.seconds = secs;
        if (infos) infos[i] = inf;
        if (inf.status == NLH_ERR_BREAKDOWN) worst = NLH_ERR_BREAKDOWN;
        else if (inf.status == NLH_ERR_NOT_CONVERGED && worst == NLH_OK)
            worst = NLH_ERR_NOT_CONVERGED;
    }
    return worst;
}

}  // namespace nlh

extern "C" nlh_status nlh_solve_batched(int nsolves, const nlh_plan *plans, const double *alphas,
                                        const double *const *b, double *const *u,
                                        const nlh_solve_opts *opts, nlh_solve_info *infos,
                                        void *stream) {
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    try {
        NLH_REQUIRE(nsolves >= 0 && (nsolves == 0 || (plans && alphas && b && u && opts)),
                    "nlh_solve_batched: NULL pointer");
        if (nsolves == 0) return NLH_OK;
        NLH_REQUIRE(opts->tol > 0.0 && opts->maxit >= 1 && opts->maxit < kMaxHist,
                    "nlh_solve_batched: tol=%g maxit=%d", opts->tol, opts->maxit);
        NLH_REQUIRE(opts->method >= NLH_CG && opts->method <= NLH_CG_DEFLATED,
                    "nlh_solve_batched: method=%d", opts->method);
        NLH_REQUIRE(opts->precond == 0 || opts->precond == 1, "nlh_solve_batched: precond=%d",
                    opts->precond);
        NLH_REQUIRE(opts->arith >= NLH_SOLVE_FP64 && opts->arith <= NLH_SOLVE_DF32,
                    "nlh_solve_batched: arith=%d", opts->arith);
        NLH_REQUIRE(opts->x0 == nullptr && opts->diag_scale == nullptr,
                    "nlh_solve_batched: x0 and diag_scale are per-solve; use nlh_solve");
        bool any_reduce = false;
        for (int i = 0; i < nsolves; ++i) {
            NLH_REQUIRE(plans[i] && b[i] && u[i], "nlh_solve_batched: NULL in solve %d", i);
            NLH_REQUIRE(alphas[i] > 0.0 && std::isfinite(alphas[i]),
                        "nlh_solve_batched: alpha[%d]=%g", i, alphas[i]);
            const int pr = plans[i]->precision;
            if (opts->arith == NLH_SOLVE_FP64)
                NLH_REQUIRE(pr & 1, "nlh_solve_batched: plan %d lacks the FP64 path", i);
            else if (opts->arith == NLH_SOLVE_DF32)
                NLH_REQUIRE(pr & 4, "nlh_solve_batched: plan %d lacks the double-float path", i);
            else
                NLH_REQUIRE((pr & 2) && (pr & 5),
                            "nlh_solve_batched: plan %d lacks the FP32 or an accurate path", i);
            any_reduce = any_reduce || plans[i]->reduce_fn != nullptr;
        }
        // one graph for the whole batch, unless a plan's matvecs call a
        // reduce callback (its collective is enqueued per call, which a
        // captured graph would not repeat): those run the round-based path
        if (!any_reduce) return solve_batched_graph(nsolves, plans, alphas, b, u, opts, infos,
                                                    (cudaStream_t)stream, t0);
        // group the solves by plan (a plan's workspace serves one solve at a time)
        std::map<nlh_plan, std::vector<int>> by_plan;
        for (int i = 0; i < nsolves; ++i) by_plan[plans[i]].push_back(i);
        std::vector<std::vector<int>> groups;
        for (auto &kv : by_plan) groups.push_back(kv.second);
        const int ns = std::min<int>((int)groups.size(), 16);
        pool_reserve(ns);
        cudaStream_t caller = (cudaStream_t)stream;
        cudaEvent_t start_ev;
        NLH_CUDA(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
        NLH_CUDA(cudaEventRecord(start_ev, caller));
        for (int k = 0; k < ns; ++k) NLH_CUDA(cudaStreamWaitEvent(g_pool[k], start_ev, 0));
        cudaEventDestroy(start_ev);

        std::vector<nlh_solve_info> inf(nsolves);
        std::vector<double> rel(nsolves, 1.0);
        std::vector<int> outer(nsolves, 0), done(nsolves, 0), status(nsolves, 1);
        std::vector<size_t> pos(groups.size(), 0);  // next solve of each group
        const bool mixed = opts->arith == NLH_SOLVE_MIXED;
        const double inner = opts->inner_tol;  // <= 0: automatic
        const int max_outer = opts->max_outer > 0 ? opts->max_outer : 20;
        while (true) {
            // one round: the current solve of every unfinished group advances one step
            std::vector<std::pair<int, int>> active;  // (group, solve)
            for (size_t gi = 0; gi < groups.size(); ++gi) {
                if (pos[gi] >= groups[gi].size()) continue;
                const int i = groups[gi][pos[gi]];
                Plan &P = *plans[i];
                cudaStream_t s = g_pool[gi % ns];
                P.stream = s;
                P.pc_kind = opts->precond;
                if (P.pc_kind == 1) ensure_pb2(P, s);
                const int accurate = (P.precision & 4) ? NLH_DF32 : NLH_FP64;
                if (!mixed) {
                    const int prec = opts->arith == NLH_SOLVE_FP64 ? NLH_FP64 : NLH_DF32;
                    krylov_launch(P, prec, alphas[i], b[i], nullptr, u[i], 0, opts->tol,
                                  opts->maxit, opts->method, nullptr, 0, s);
                    residual_launch(P, prec, alphas[i], b[i], u[i], nullptr, s);
                } else {
                    if (outer[i] == 0) {
                        NLH_CUDA(cudaMemsetAsync(u[i], 0, sizeof(double) * P.N, s));
                        NLH_CUDA(cudaMemcpyAsync(P.rhs, b[i], sizeof(double) * P.N,
                                                 cudaMemcpyDeviceToDevice, s));
                    }
                    krylov_launch(P, NLH_FP32, alphas[i], P.rhs, nullptr, u[i], 1,
                                  inner_tolerance(inner, opts->tol, rel[i]), opts->maxit,
                                  opts->method, nullptr, 0, s, inner <= 0 ? kInnerStag : 0);
                    residual_launch(P, accurate, alphas[i], b[i], u[i], P.rhs, s);
                }
                active.push_back({(int)gi, i});
            }
            if (active.empty()) break;
            for (int k = 0; k < ns; ++k) NLH_CUDA(cudaStreamSynchronize(g_pool[k]));
            for (auto &a : active) {
                const int gi = a.first, i = a.second;
                Plan &P = *plans[i];
                KrylovResult kr = krylov_collect(P);
                const double r = residual_collect(P);
                inf[i].iters += kr.iters;
                ++outer[i];
                if (!mixed) {
                    inf[i].matvecs_fp64 += kr.matvecs + 1;
                    inf[i].rel_res = kr.rel;
                    status[i] = kr.status;
                    done[i] = 1;
                } else {
                    inf[i].matvecs_fp32 += kr.matvecs;
                    inf[i].matvecs_fp64 += 1;
                    inf[i].rel_res = r;
                    rel[i] = r;
                    if (kr.status == -4) {
                        status[i] = -4;
                        done[i] = 1;
                    } else if (r <= opts->tol) {
                        status[i] = 0;
                        done[i] = 1;
                    } else if (outer[i] >= max_outer) {
                        status[i] = 1;
                        done[i] = 1;
                    }
                }
                inf[i].rel_res_true = r;
                inf[i].outer = outer[i];
                if (done[i]) ++pos[gi];
            }
        }
        for (int k = 0; k < ns; ++k) {
            NLH_CUDA(cudaEventRecord(g_pool_ev[k], g_pool[k]));
            NLH_CUDA(cudaStreamWaitEvent(caller, g_pool_ev[k], 0));
        }
        for (int i = 0; i < nsolves; ++i) check_device_error(*plans[i], g_pool[0]);
        const double secs =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        nlh_status worst = NLH_OK;
        for (int i = 0; i < nsolves; ++i) {
            inf[i].status = status[i] == 0 ? NLH_OK
                                           : (status[i] == -4 ? NLH_ERR_BREAKDOWN
                                                              : NLH_ERR_NOT_CONVERGED);
            inf[i].seconds = secs;
            if (infos) infos[i] = inf[i];
            if (inf[i].status == NLH_ERR_BREAKDOWN) worst = NLH_ERR_BREAKDOWN;
            else if (inf[i].status == NLH_ERR_NOT_CONVERGED && worst == NLH_OK)
                worst = NLH_ERR_NOT_CONVERGED;
        }
        return worst;
    } catch (Failure &f) {
        return f.st;
    }
}

// Test hooks (include/nlh_selftest.h): the host side of the solver's
// stopping rules, callable without a GPU.
extern "C" double nlh_selftest_inner_tolerance(double inner, double tol, double rel) {
    return nlh::inner_tolerance(inner, tol, rel);
}

extern "C" int nlh_selftest_convergence(const double *rel, int n, double tol, int maxit,
                                        int stag) {
    if (!rel || n < 0) return -2;
    nlh::SolveState st{};
    st.tol = tol;
    st.maxit = maxit;
    st.stag = stag;
    for (int k = 0; k < n; ++k) {
        nlh::convergence_step(&st, rel[k], k);
        if (st.done) return k;
    }
    return -1;
}
