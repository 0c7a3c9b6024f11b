// mis.cu -- feature windows ranked by mutual information (Sec. 5; the
// estimator and its conventions are stated in include/nlh_mis.h).
//
// Kernels, all reading the image (FP64, L2-resident for the sizes of the
// method) and forming the patch dimensions on the fly:
//   k_mis_range       per-(slice of rows, variable) minimum and maximum as
//                     order-preserving int64 keys (no FP64 instructions);
//                     variable D is the target f itself, 0..D-1 the patch
//                     dimensions
//   k_mis_range_final the slices' extrema -> lo and bins / (hi - lo), their
//                     FP32 roundings and the FP32 fast path's error margin
//   k_mis_prep        the image rounded to FP32 and the target's bins
//                     (exact, FP64), once per pixel
//   k_mis_hist        the joint (feature bin, target bin) histogram of one
//                     patch dimension per blockIdx.y in shared memory
//                     (integer atomics, one per distinct cell per warp:
//                     exact, order-free), added to the global counts once
//                     per block.  The feature bin comes from the FP32 image
//                     when the FP32 value is clear of the bin edges by a
//                     proven margin (then it equals the FP64 decision), and
//                     from the exact FP64 formula otherwise (GB300's FP64
//                     rate is 1/64 of FP32)
//   k_mis_score       one block per dimension: marginals, then the plug-in
//                     mutual information in a fixed-order reduction
//   k_mis_rank        ranks (MIS descending, ties to the lower dimension)
//                     and the windows as ranked triples
#include "common.cuh"
#include "../../include/nlh_mis.h"

#include <algorithm>
#include <climits>

namespace nlh {
namespace {

constexpr int kMT = 256;          // threads of the reductions / histograms
constexpr int kMaxSlices = 64;    // range slices per variable
constexpr int kMaxBins = 128;
constexpr int kMaxRadius = 6;     // D <= 169, L <= 57

struct Img {
    const double *x;
    const float *x32;  // the image rounded to FP32 (fast path of the bins)
    int n1, n2, rho, pad;
};

// Source pixel of patch dimension k at (r, c) in one axis: the offset
// position, reflected, or -1 outside the image with zero padding
// (the nlh_patch_features convention k = (dr + rho)(2 rho + 1) + (dc + rho)).
__device__ __forceinline__ int src_axis(int p, int off, int n, int pad) {
    const int q = p + off;
    if (q >= 0 && q < n) return q;
    return pad == 0 ? -1 : reflect_index(q, n);
}

// Order-preserving int64 key of a double (so that min / max run on the
// integer pipes; -0.0 sorts just below +0.0, which is equal as a value).
__device__ __forceinline__ long long okey(double v) {
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double from_okey(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL));
}

// Exact equal-width bin: the difference and the product rounded separately
// in FP64 (no contraction), inv = 0 marks a constant variable.  t is in
// [0, bins] for finite input; the comparisons also keep a NaN in range.
__device__ __forceinline__ int bin_of(double x, double lo, double inv, int bins) {
    if (inv == 0.0) return 0;
    const double t = __dmul_rn(__dsub_rn(x, lo), inv);
    if (!(t >= 0.0)) return 0;
    return t < (double)(bins - 1) ? (int)t : bins - 1;
}

// Grid (slices, D + 1): block (s, v) covers rows s, s + slices, ... of
// variable v; min / max as order keys.
__global__ void __launch_bounds__(kMT) k_mis_range(Img g, int D, long long *__restrict__ part) {
    __shared__ long long smin[kMT], smax[kMT];
    const int var = blockIdx.y, G = gridDim.x;
    const int P = 2 * g.rho + 1;
    const int dr = var < D ? var / P - g.rho : 0, dc = var < D ? var % P - g.rho : 0;
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int r = blockIdx.x; r < g.n1; r += G) {
        const int rr = src_axis(r, dr, g.n1, g.pad);
        for (int c = threadIdx.x; c < g.n2; c += blockDim.x) {
            const int cc = src_axis(c, dc, g.n2, g.pad);
            const double v = (rr < 0 || cc < 0) ? 0.0 : g.x[(int64_t)rr * g.n2 + cc];
            const long long k = okey(v);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            smin[threadIdx.x] = min(smin[threadIdx.x], smin[threadIdx.x + h]);
            smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * ((int64_t)var * G + blockIdx.x)] = smin[0];
        part[2 * ((int64_t)var * G + blockIdx.x) + 1] = smax[0];
    }
}

// Per variable (patch dimensions 0..D-1, the image itself D):
//   bp[4 v + 0] = lo, bp[4 v + 1] = inv = bins / (hi - lo) (0 if constant),
//   bp[4 v + 2] = lo and bp[4 v + 3] = inv rounded to FP32 for the fast path,
//   margin[v] = a bound on |t32 - t| (t = (x - lo) inv exactly, t32 the FP32
//   evaluation from the FP32-rounded x, lo, inv): a fast-path value farther
//   than the margin from every integer has the exact bin (and a margin >=
//   0.25 disables the fast path).
__global__ void k_mis_range_final(const long long *__restrict__ part, int G, int bins,
                                  double *__restrict__ bp, float *__restrict__ margin) {
    if (threadIdx.x != 0) return;
    const int var = blockIdx.x;
    long long klo = LLONG_MAX, khi = LLONG_MIN;
    for (int s = 0; s < G; ++s) {
        klo = min(klo, part[2 * ((int64_t)var * G + s)]);
        khi = max(khi, part[2 * ((int64_t)var * G + s) + 1]);
    }
    const double lo = from_okey(klo), hi = from_okey(khi);
    const double inv = hi > lo ? __ddiv_rn((double)bins, __dsub_rn(hi, lo)) : 0.0;
    bp[4 * var] = lo;
    bp[4 * var + 1] = inv;
    bp[4 * var + 2] = (double)(float)lo;
    bp[4 * var + 3] = (double)(float)inv;
    // |t32 - t| <= inv (|x - xf| + |lo - lo32|) (1 + 2u) + |t| 3u + 2u |t|,
    // u = 2^-24, |x|, |lo| <= A = max(|lo|, |hi|), |t| <= bins: bounded by
    // 4u (2 A inv + 2 bins); doubled for safety.  Non-finite -> slow path.
    const double u = 5.9604644775390625e-08;
    const double A = fmax(fabs(lo), fabs(hi));
    const double m = 8.0 * u * (2.0 * A * inv + 2.0 * bins);
    margin[var] = (isfinite(m) && m < 0.25) ? (float)m : 1.0f;
}

// x32 = x rounded to FP32, tb = the exact bin of the image itself (the
// target variable D), once per pixel.
__global__ void __launch_bounds__(kMT) k_mis_prep(const double *__restrict__ x, int64_t N,
                                                  const double *__restrict__ bp, int D, int bins,
                                                  float *__restrict__ x32,
                                                  unsigned char *__restrict__ tb) {
    const double lo = bp[4 * D], inv = bp[4 * D + 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        x32[i] = (float)v;
        tb[i] = (unsigned char)bin_of(v, lo, inv, bins);
    }
}

// Grid (slices, D): block (s, d) adds rows s, s + slices, ... of dimension
// d into a shared histogram; lanes of a warp with the same cell add once
// (correlated dimensions crowd the diagonal).
__global__ void __launch_bounds__(kMT) k_mis_hist(Img g, int bins, const double *__restrict__ bp,
                                                  const float *__restrict__ margin,
                                                  const unsigned char *__restrict__ tb,
                                                  int *__restrict__ counts) {
    extern __shared__ int sh[];
    const int d = blockIdx.y;
    const int nb2 = bins * bins;
    for (int j = threadIdx.x; j < nb2; j += blockDim.x) sh[j] = 0;
    __syncthreads();
    const int P = 2 * g.rho + 1;
    const int dr = d / P - g.rho, dc = d % P - g.rho;
    const double *p = bp + 4 * d;
    const float mg = margin[d];
    const int lane = threadIdx.x & 31;
    for (int r = blockIdx.x; r < g.n1; r += gridDim.x) {
        const int rr = src_axis(r, dr, g.n1, g.pad);
        for (int c0 = 0; c0 < g.n2; c0 += blockDim.x) {
            const int c = c0 + threadIdx.x;
            const bool in = c < g.n2;
            int key = 0;
            if (in) {
                const int cc = src_axis(c, dc, g.n2, g.pad);
                int a;
                if (rr < 0 || cc < 0) {
                    a = bin_of(0.0, p[0], p[1], bins);  // zero padding
                } else {
                    const int64_t src = (int64_t)rr * g.n2 + cc;
                    a = -1;
                    if (p[1] == 0.0) {
                        a = 0;
                    } else if (mg < 0.25f) {
                        // FP32 evaluation; its bin is exact when t lies
                        // farther than the margin from every bin edge
                        const float t = (g.x32[src] - (float)p[2]) * (float)p[3];
                        const float fl = floorf(t);
                        if (t >= mg && t < (float)(bins - 1) - mg && t - fl >= mg &&
                            fl + 1.0f - t >= mg)
                            a = (int)fl;
                        else if (t >= (float)(bins - 1) + mg)
                            a = bins - 1;
                    }
                    if (a < 0) a = bin_of(g.x[src], p[0], p[1], bins);  // exact
                }
                key = a * bins + tb[(int64_t)r * g.n2 + c];
            }
            const unsigned act = __ballot_sync(0xffffffffu, in);
            if (in) {
                const unsigned peers = __match_any_sync(act, key);
                if (lane == __ffs(peers) - 1) atomicAdd(&sh[key], __popc(peers));
            }
        }
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
        // slices of rows: about four blocks per SM over all variables
        int G = (4 * 152 + D) / (D + 1);
        G = std::max(1, std::min({G, kMaxSlices, n1}));
        const size_t nb2 = (size_t)bins * bins;
        // scratch: range partials (int64 keys), bin parameters, margins,
        // the FP32 image, the target bins, and the counts if not given
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t at = off;
            off += (bytes + 255) / 256 * 256;
            return at;
        };
        const size_t o_part = take(2 * (size_t)(D + 1) * G * sizeof(long long));
        const size_t o_bp = take(4 * (size_t)(D + 1) * sizeof(double));
        const size_t o_mg = take((size_t)(D + 1) * sizeof(float));
        const size_t o_x32 = take((size_t)N * sizeof(float));
        const size_t o_tb = take((size_t)N);
        const size_t o_cnt = counts ? 0 : take(nb2 * D * sizeof(int));
        unsigned char *scratch = nullptr;
        NLH_CUDA(cudaMallocAsync((void **)&scratch, off, s));
        long long *part = reinterpret_cast<long long *>(scratch + o_part);
        double *bp = reinterpret_cast<double *>(scratch + o_bp);
        float *mg = reinterpret_cast<float *>(scratch + o_mg);
        float *x32 = reinterpret_cast<float *>(scratch + o_x32);
        unsigned char *tb = scratch + o_tb;
        int *cnt = counts ? counts : reinterpret_cast<int *>(scratch + o_cnt);
        const Img g{image, x32, n1, n2, radius, pad};
        NLH_CUDA(cudaMemsetAsync(cnt, 0, nb2 * D * sizeof(int), s));
        k_mis_range<<<dim3(G, D + 1), kMT, 0, s>>>(g, D, part);
        NLH_CHECK_LAUNCH();
        k_mis_range_final<<<D + 1, 32, 0, s>>>(part, G, bins, bp, mg);
        NLH_CHECK_LAUNCH();
        k_mis_prep<<<(int)std::min<int64_t>((N + kMT - 1) / kMT, 8 * 152), kMT, 0, s>>>(
            image, N, bp, D, bins, x32, tb);
        NLH_CHECK_LAUNCH();
        // histograms: about eight blocks per SM over the D dimensions
        int GH = (8 * 152 + D - 1) / D;
        GH = std::max(1, std::min(GH, n1));
        const int hsm = (int)(nb2 * sizeof(int));
        if (hsm > 48 * 1024)
            NLH_CUDA(cudaFuncSetAttribute(k_mis_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          hsm));
        k_mis_hist<<<dim3(GH, D), kMT, hsm, s>>>(g, bins, bp, mg, tb, cnt);
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
