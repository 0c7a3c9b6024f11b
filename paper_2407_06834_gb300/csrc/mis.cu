// mis.cu -- feature windows ranked by mutual information (Sec. 5; the
// estimator and its conventions are stated in include/nlh_mis.h).
//
// Kernels, all reading the image (FP64, L2-resident for the sizes of the
// method) and forming the patch dimensions on the fly:
//   k_mis_range       per-(slice, variable) minimum and maximum; variable D
//                     is the target f itself, 0..D-1 the patch dimensions
//   k_mis_range_final the slices' extrema -> lo and bins / (hi - lo)
//   k_mis_hist        the joint (feature bin, target bin) histogram of one
//                     patch dimension per blockIdx.y in shared memory
//                     (integer atomics: exact, order-free), added to the
//                     global counts once per block
//   k_mis_score       one block per dimension: marginals, then the plug-in
//                     mutual information in a fixed-order reduction
//   k_mis_rank        ranks (MIS descending, ties to the lower dimension)
//                     and the windows as ranked triples
#include "common.cuh"
#include "../../include/nlh_mis.h"

#include <algorithm>

namespace nlh {
namespace {

constexpr int kMT = 256;          // threads of the reductions / histograms
constexpr int kMaxSlices = 64;    // range slices per variable
constexpr int kMaxBins = 128;
constexpr int kMaxRadius = 6;     // D <= 169, L <= 57

struct Img {
    const double *x;
    int n1, n2, rho, pad;
};

// Patch dimension k of pixel i (the nlh_patch_features convention:
// k = (dr + rho)(2 rho + 1) + (dc + rho)).
__device__ __forceinline__ double feature(const Img &g, int64_t i, int k) {
    const int P = 2 * g.rho + 1;
    const int r = (int)(i / g.n2), c = (int)(i - (int64_t)r * g.n2);
    const int rr = r + k / P - g.rho, cc = c + k % P - g.rho;
    if (g.pad == 0)
        return (rr < 0 || rr >= g.n1 || cc < 0 || cc >= g.n2) ? 0.0 : g.x[(int64_t)rr * g.n2 + cc];
    return g.x[(int64_t)reflect_index(rr, g.n1) * g.n2 + reflect_index(cc, g.n2)];
}

__device__ __forceinline__ double value(const Img &g, int64_t i, int var, int D) {
    return var == D ? g.x[i] : feature(g, i, var);
}

// Equal-width bin: the difference and the product rounded separately
// (no contraction), inv = 0 marks a constant variable.  t is in [0, bins]
// for finite input; the comparisons also keep a NaN (bin 0) in range.
__device__ __forceinline__ int bin_of(double x, double lo, double inv, int bins) {
    if (inv == 0.0) return 0;
    const double t = __dmul_rn(__dsub_rn(x, lo), inv);
    if (!(t >= 0.0)) return 0;
    return t < (double)(bins - 1) ? (int)t : bins - 1;
}

__global__ void __launch_bounds__(kMT) k_mis_range(Img g, int D, double *__restrict__ part) {
    __shared__ double smin[kMT], smax[kMT];
    const int var = blockIdx.y, G = gridDim.x;
    const int64_t N = (int64_t)g.n1 * g.n2;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)G * blockDim.x) {
        const double v = value(g, i, var, D);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + h]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * ((int64_t)var * G + blockIdx.x)] = smin[0];
        part[2 * ((int64_t)var * G + blockIdx.x) + 1] = smax[0];
    }
}

// lohi[2 var] = lo, lohi[2 var + 1] = bins / (hi - lo) (0 if hi = lo).
__global__ void k_mis_range_final(const double *__restrict__ part, int G, int bins,
                                  double *__restrict__ lohi) {
    if (threadIdx.x != 0) return;
    const int var = blockIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    for (int s = 0; s < G; ++s) {
        lo = fmin(lo, part[2 * ((int64_t)var * G + s)]);
        hi = fmax(hi, part[2 * ((int64_t)var * G + s) + 1]);
    }
    lohi[2 * var] = lo;
    lohi[2 * var + 1] = hi > lo ? __ddiv_rn((double)bins, __dsub_rn(hi, lo)) : 0.0;
}

__global__ void __launch_bounds__(kMT) k_mis_hist(Img g, int D, int bins,
                                                  const double *__restrict__ lohi,
                                                  int *__restrict__ counts) {
    extern __shared__ int sh[];
    const int d = blockIdx.y;
    const int nb2 = bins * bins;
    for (int j = threadIdx.x; j < nb2; j += blockDim.x) sh[j] = 0;
    __syncthreads();
    const double flo = lohi[2 * d], finv = lohi[2 * d + 1];
    const double ylo = lohi[2 * D], yinv = lohi[2 * D + 1];
    const int64_t N = (int64_t)g.n1 * g.n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = bin_of(feature(g, i, d), flo, finv, bins);
        const int b = bin_of(g.x[i], ylo, yinv, bins);
        atomicAdd(&sh[a * bins + b], 1);
    }
    __syncthreads();
    int *out = counts + (int64_t)d * nb2;
    for (int j = threadIdx.x; j < nb2; j += blockDim.x)
        if (sh[j]) atomicAdd(&out[j], sh[j]);
}

__global__ void __launch_bounds__(kMT) k_mis_score(const int *__restrict__ counts, int bins,
                                                   int64_t N, double *__restrict__ mis) {
    __shared__ int ca[kMaxBins], cb[kMaxBins];
    __shared__ double red[kMT];
    const int d = blockIdx.x;
    const int *c = counts + (int64_t)d * bins * bins;
    for (int a = threadIdx.x; a < bins; a += blockDim.x) {
        int s = 0, t = 0;
        for (int b = 0; b < bins; ++b) {
            s += c[a * bins + b];
            t += c[b * bins + a];
        }
        ca[a] = s;
        cb[a] = t;
    }
    __syncthreads();
    const double n = (double)N;
    double acc = 0.0;
    for (int j = threadIdx.x; j < bins * bins; j += blockDim.x) {
        const int cab = c[j];
        if (cab > 0) {
            const double v = (double)cab;
            const double q = (v * n) / ((double)ca[j / bins] * (double)cb[j % bins]);
            acc += (v / n) * log(q);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) mis[d] = red[0];
}

__global__ void __launch_bounds__(kMT) k_mis_rank(const double *__restrict__ mis, int D, int L,
                                                  int32_t *__restrict__ windows) {
    const int t = threadIdx.x;
    if (t < D) {
        const double m = mis[t];
        int r = 0;
        for (int e = 0; e < D; ++e) {
            const double o = mis[e];
            r += (o > m || (o == m && e < t)) ? 1 : 0;
        }
        windows[r] = t;
    } else if (t < 3 * L) {
        windows[t] = -1;
    }
}

}  // namespace
}  // namespace nlh

using namespace nlh;

extern "C" {

nlh_status nlh_mis_windows(const double *image, int n1, int n2, int radius, int pad, int bins,
                           double *mis, int32_t *windows, int32_t *counts, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(image && mis, "nlh_mis_windows: NULL image or mis");
        NLH_REQUIRE(n1 >= 1 && n2 >= 1 && (int64_t)n1 * n2 < ((int64_t)1 << 31),
                    "nlh_mis_windows: bad image size %d x %d", n1, n2);
        NLH_REQUIRE(radius >= 0 && radius <= kMaxRadius, "nlh_mis_windows: radius=%d not in 0..%d",
                    radius, kMaxRadius);
        NLH_REQUIRE(pad == 0 || pad == 1, "nlh_mis_windows: pad must be 0 or 1");
        NLH_REQUIRE(bins >= 2 && bins <= kMaxBins, "nlh_mis_windows: bins=%d not in 2..%d", bins,
                    kMaxBins);
        cudaStream_t s = (cudaStream_t)stream;
        const int D = (2 * radius + 1) * (2 * radius + 1);
        const int L = (D + 2) / 3;
        const int64_t N = (int64_t)n1 * n2;
        const Img g{image, n1, n2, radius, pad};
        // slices: about four blocks per SM over all variables, 2048+ pixels each
        int G = (int)std::min<int64_t>((4 * 152 + D) / (D + 1), (N + 2047) / 2048);
        G = std::max(1, std::min(G, kMaxSlices));
        const size_t nb2 = (size_t)bins * bins;
        double *scratch = nullptr;
        const size_t ndbl = 2 * (size_t)(D + 1) * G + 2 * (size_t)(D + 1);
        const size_t bytes = ndbl * sizeof(double) + (counts ? 0 : nb2 * D * sizeof(int));
        NLH_CUDA(cudaMallocAsync((void **)&scratch, bytes, s));
        double *part = scratch, *lohi = scratch + 2 * (size_t)(D + 1) * G;
        int *cnt = counts ? counts : reinterpret_cast<int *>(scratch + ndbl);
        NLH_CUDA(cudaMemsetAsync(cnt, 0, nb2 * D * sizeof(int), s));
        k_mis_range<<<dim3(G, D + 1), kMT, 0, s>>>(g, D, part);
        NLH_CHECK_LAUNCH();
        k_mis_range_final<<<D + 1, 32, 0, s>>>(part, G, bins, lohi);
        NLH_CHECK_LAUNCH();
        // histograms: about eight blocks per SM over the D dimensions
        int GH = (int)std::min<int64_t>((8 * 152 + D - 1) / D, (N + 4095) / 4096);
        GH = std::max(1, GH);
        const int hsm = (int)(nb2 * sizeof(int));
        if (hsm > 48 * 1024)
            NLH_CUDA(cudaFuncSetAttribute(k_mis_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          hsm));
        k_mis_hist<<<dim3(GH, D), kMT, hsm, s>>>(g, D, bins, lohi, cnt);
        NLH_CHECK_LAUNCH();
        k_mis_score<<<D, kMT, 0, s>>>(cnt, bins, N, mis);
        NLH_CHECK_LAUNCH();
        if (windows) {
            k_mis_rank<<<1, kMT, 0, s>>>(mis, D, L, windows);
            NLH_CHECK_LAUNCH();
        }
        NLH_CUDA(cudaFreeAsync(scratch, s));
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

}  // extern "C"
