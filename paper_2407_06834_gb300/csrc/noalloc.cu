// noalloc.cu -- residual norms without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: code running while a framework captures a CUDA graph (where a
// cudaMalloc is not allowed), real-time loops that must not pay allocation
// latency, or processes whose device memory is entirely owned by another
// allocator.  nlh_residual_norms_noalloc serves them: it is the same
// deterministic two-pass reduction that the solver uses for its final
// residual (||b - q||, ||b||), but its per-block partial sums live in a
// fixed array of this library instead of plan memory, and the call makes no
// allocation of any kind.
#include "common.cuh"

#include <mutex>

namespace nlh {

// Per-block partial sums (2 doubles per block).  Each block of a call writes
// its own two slots before the finishing kernel reads them, so nothing has to
// start at zero; the contents of one call survive until the next call.
constexpr int kNoAllocChunk = 4096;          // elements reduced per block
constexpr int kNoAllocMaxBlocks = 8192;      // 128 KiB of partials
constexpr int64_t kNoAllocMaxN = (int64_t)kNoAllocChunk * kNoAllocMaxBlocks;
static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxBlocks];

__global__ void __launch_bounds__(kRedThreads)
k_residual_chunks(const double *__restrict__ b, const double *__restrict__ q, int64_t N,
                  double *__restrict__ res, double *__restrict__ partials) {
    __shared__ double sh[33];
    const int64_t base = (int64_t)blockIdx.x * kNoAllocChunk;
    const int64_t end = base + kNoAllocChunk < N ? base + kNoAllocChunk : N;
    double s_rr = 0, s_bb = 0;
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
        double bi = b[i], ri = bi - q[i];
        if (res) res[i] = ri;
        s_rr = fma(ri, ri, s_rr);
        s_bb = fma(bi, bi, s_bb);
    }
    double v0 = block_sum(s_rr, sh), v1 = block_sum(s_bb, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x + 0] = v0;
        partials[2 * blockIdx.x + 1] = v1;
    }
}

__global__ void __launch_bounds__(kRedThreads)
k_residual_finish(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
    __shared__ double sh[33];
    double rr = reduce_partials(partials, nblocks, 2, 0, sh);
    double bb = reduce_partials(partials, nblocks, 2, 1, sh);
    if (threadIdx.x == 0) {
        out[0] = sqrt(rr);
        out[1] = sqrt(bb);
    }
}

// Device address of the partials array on the current device.  Outside
// stream capture it is looked up afresh on every call (cudaGetSymbolAddress
// allocates nothing), so that a device reset or a new primary context never
// leaves a stale address behind; the last address seen per device is kept
// for calls made while `stream` is being captured, where the lookup itself
// may not be issued.  A first call on a device during capture is an error.
static double *noalloc_partials_ptr(cudaStream_t stream) {
    static std::mutex mu;
    static double *cache[64] = {nullptr};
    int dev = 0;
    NLH_CUDA(cudaGetDevice(&dev));
    NLH_REQUIRE(dev >= 0 && dev < 64, "nlh_residual_norms_noalloc: device %d unsupported", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NLH_CUDA(cudaStreamIsCapturing(stream, &cap));
    std::lock_guard<std::mutex> lk(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *ptr = nullptr;
        NLH_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_partials));
        cache[dev] = static_cast<double *>(ptr);
    }
    NLH_REQUIRE(cache[dev],
                "nlh_residual_norms_noalloc: the first call on a device must come before any "
                "stream capture");
    return cache[dev];
}

}  // namespace nlh

extern "C" nlh_status nlh_residual_norms_noalloc(const double *b, const double *q, int64_t N,
                                                 double *res, double *norms, void *stream) {
    nlh::clear_error();
    try {
        NLH_REQUIRE(b && q && norms, "nlh_residual_norms_noalloc: NULL pointer");
        NLH_REQUIRE(N >= 1, "nlh_residual_norms_noalloc: N=%lld must be >= 1", (long long)N);
        NLH_REQUIRE(N <= nlh::kNoAllocMaxN,
                    "nlh_residual_norms_noalloc: N=%lld exceeds the maximum %lld of the fixed "
                    "scratch array",
                    (long long)N, (long long)nlh::kNoAllocMaxN);
        cudaStream_t s = (cudaStream_t)stream;
        double *partials = nlh::noalloc_partials_ptr(s);
        const int nblocks = nlh::div_up(N, nlh::kNoAllocChunk);
        nlh::k_residual_chunks<<<nblocks, nlh::kRedThreads, 0, s>>>(b, q, N, res, partials);
        NLH_CHECK_LAUNCH();
        nlh::k_residual_finish<<<1, nlh::kRedThreads, 0, s>>>(partials, nblocks, norms);
        NLH_CHECK_LAUNCH();
        return NLH_OK;
    } catch (nlh::Failure &f) {
        return f.st;
    }
}
