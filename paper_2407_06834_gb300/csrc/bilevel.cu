// bilevel.cu -- reductions of the bilevel learning of alpha (Sec. 2 and
// Sec. 5.5): the misfit ||u - u_c||^2 with the adjoint right-hand side
// u - u_c, and the gradient term <p, f - u>.  Two-stage fixed-order sums.
#include "common.cuh"
#include "../../include/nlh_bilevel.h"

namespace nlh {
namespace {

constexpr int kBT = 256, kBB = 304;  // threads, blocks (2 per SM)

__device__ __forceinline__ double block_reduce(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(kBT) k_misfit(const double *__restrict__ u,
                                                const double *__restrict__ uc, int64_t N,
                                                double *__restrict__ r,
                                                double *__restrict__ part) {
    __shared__ double sh[kBT];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = u[i] - uc[i];
        if (r) r[i] = d;
        acc = fma(d, d, acc);
    }
    const double s = block_reduce(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kBT) k_grad_term(const double *__restrict__ p,
                                                   const double *__restrict__ f,
                                                   const double *__restrict__ u, int64_t N,
                                                   double *__restrict__ part) {
    __shared__ double sh[kBT];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(p[i], f[i] - u[i], acc);
    const double s = block_reduce(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kBT) k_final(const double *__restrict__ part, int n,
                                               double *__restrict__ out) {
    __shared__ double sh[kBT];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    const double s = block_reduce(acc, sh);
    if (threadIdx.x == 0) *out = s;
}

// Scratch for the partial sums, from the stream-ordered pool (so that calls
// on different streams never share it).
double *scratch(cudaStream_t s) {
    double *b = nullptr;
    NLH_CUDA(cudaMallocAsync(&b, sizeof(double) * (kBB + 1), s));
    return b;
}

double finish(double *part, cudaStream_t s) {
    k_final<<<1, kBT, 0, s>>>(part, kBB, part + kBB);
    NLH_CHECK_LAUNCH();
    double out = 0.0;
    NLH_CUDA(cudaMemcpyAsync(&out, part + kBB, sizeof(double), cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaFreeAsync(part, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    return out;
}

}  // namespace
}  // namespace nlh

using namespace nlh;

extern "C" {

nlh_status nlh_bilevel_misfit(int64_t N, const double *u, const double *uc, double *r,
                              double *sq, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(u && uc && sq && N >= 1, "nlh_bilevel_misfit: bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        double *part = scratch(s);
        k_misfit<<<kBB, kBT, 0, s>>>(u, uc, N, r, part);
        NLH_CHECK_LAUNCH();
        *sq = finish(part, s);
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_bilevel_gradient_term(int64_t N, const double *p, const double *f,
                                     const double *u, double *dot, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(p && f && u && dot && N >= 1, "nlh_bilevel_gradient_term: bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        double *part = scratch(s);
        k_grad_term<<<kBB, kBT, 0, s>>>(p, f, u, N, part);
        NLH_CHECK_LAUNCH();
        *dot = finish(part, s);
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

}  // extern "C"
