// nfft.cu -- the per-matvec NFFT fast Gauss transform (Sec. 3 of arXiv
// 2407.06834): for every window l,
//   spread   G_l[g] = sum_i v_i prod_d phi(g_d/n - x~_{i,d})      (adjoint NFFT
//                                                                 gridding)
//   convolve G'_l = IFFT(w .* FFT(G_l)) per axis (w: Gaussian coefficients
//            over the squared window transform, |k| < M/2)
//   interp   y_{l,i} = sum_g G'_l[g] prod_d phi(x~_{i,d} - g_d/n)  (NFFT)
// and the epilogue y = (1/L) sum_l y_l  (= Gamma_full v), optionally
// L v = d o v - y or (alpha I + L) v, fused with the dot x^T y for CG.
//
// Work decomposition: points are sorted by grid cell; a work item is up to
// kmax points of one cell, which share one 2m x 2m x 2m stencil.  One CTA
// per item keeps the item's stencil (spreading accumulators or interpolation
// grid values) in registers, so the inner loop is pure FMA: no atomics per
// point.  Spreading flushes each item's accumulators with one atomic add per
// stencil cell.
#include "common.cuh"

namespace nlh {

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C> __device__ __forceinline__ C cshfl(C a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)};
}

constexpr int kChunk = 32;  // points staged in shared memory at a time

// ------------------------------------------------------------------ spreading
template <typename T, int W2, int NW>
__global__ void __launch_bounds__(32 * NW)
k_spread(const int4 *__restrict__ items, const int *__restrict__ perm,
         const T *__restrict__ wts, const double *__restrict__ v, T *__restrict__ grid, int n,
         int m, const int *__restrict__ done) {
    constexpr int NT = 32 * NW, NP = W2 * W2, PPT = (NP + NT - 1) / NT, PW = 3 * W2;
    __shared__ T sw[kChunk * PW];
    __shared__ T sv[kChunk];
    if (done && *done) return;
    const int4 it = items[blockIdx.x];
    const int l = it.x, cell = it.y, start = it.z, cnt = it.w;
    const int tid = threadIdx.x;
    int bb[PPT], cc[PPT];
    bool ok[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int p = tid + NT * k;
        ok[k] = p < NP;
        bb[k] = ok[k] ? p % W2 : 0;
        cc[k] = ok[k] ? p / W2 : 0;
    }
    T acc[PPT][W2];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
        for (int a = 0; a < W2; ++a) acc[k][a] = T(0);

    for (int c0 = 0; c0 < cnt; c0 += kChunk) {
        const int cn = min(kChunk, cnt - c0);
        const T *src = wts + (int64_t)(start + c0) * PW;
        for (int e = tid; e < cn * PW; e += NT) sw[e] = src[e];
        for (int e = tid; e < cn; e += NT) sv[e] = (T)v[perm[start + c0 + e]];
        __syncthreads();
        for (int j = 0; j < cn; ++j) {
            const T *wp = sw + j * PW;
            T wx[W2];
#pragma unroll
            for (int a = 0; a < W2; ++a) wx[a] = wp[a];
            const T vj = sv[j];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (ok[k]) {
                    T s = vj * wp[W2 + bb[k]] * wp[2 * W2 + cc[k]];
#pragma unroll
                    for (int a = 0; a < W2; ++a) acc[k][a] = fma(s, wx[a], acc[k][a]);
                }
            }
        }
        __syncthreads();
    }
    const int msk = n - 1;
    const int x0 = cell % n, y0 = (cell / n) % n, z0 = cell / (n * n);
    T *g = grid + (int64_t)l * n * n * n;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!ok[k]) continue;
        int y = (y0 - m + 1 + bb[k]) & msk, z = (z0 - m + 1 + cc[k]) & msk;
        T *row = g + ((int64_t)z * n + y) * n;
#pragma unroll
        for (int a = 0; a < W2; ++a) atomicAdd(&row[(x0 - m + 1 + a) & msk], acc[k][a]);
    }
}

// ------------------------------------------------------------------ interpolation
template <typename T, int W2, int NW>
__global__ void __launch_bounds__(32 * NW)
k_interp(const int4 *__restrict__ items, const int *__restrict__ perm,
         const T *__restrict__ wts, const T *__restrict__ grid, double *__restrict__ Y, int n,
         int m, int64_t N, const int *__restrict__ done) {
    constexpr int NT = 32 * NW, NP = W2 * W2, PPT = (NP + NT - 1) / NT, PW = 3 * W2;
    __shared__ T sw[kChunk * PW];
    __shared__ T sred[kChunk];
    if (done && *done) return;
    const int4 it = items[blockIdx.x];
    const int l = it.x, cell = it.y, start = it.z, cnt = it.w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int msk = n - 1;
    const int x0 = cell % n, y0 = (cell / n) % n, z0 = cell / (n * n);
    const T *g = grid + (int64_t)l * n * n * n;
    int bb[PPT], cc[PPT];
    bool ok[PPT];
    T H[PPT][W2];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int p = tid + NT * k;
        ok[k] = p < NP;
        bb[k] = ok[k] ? p % W2 : 0;
        cc[k] = ok[k] ? p / W2 : 0;
        int y = (y0 - m + 1 + bb[k]) & msk, z = (z0 - m + 1 + cc[k]) & msk;
        const T *row = g + ((int64_t)z * n + y) * n;
#pragma unroll
        for (int a = 0; a < W2; ++a) H[k][a] = ok[k] ? row[(x0 - m + 1 + a) & msk] : T(0);
    }
    for (int c0 = 0; c0 < cnt; c0 += kChunk) {
        const int cn = min(kChunk, cnt - c0);
        const T *src = wts + (int64_t)(start + c0) * PW;
        for (int e = tid; e < cn * PW; e += NT) sw[e] = src[e];
        __syncthreads();
        T part[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            T sum = T(0);
            if (j < cn) {
                const T *wp = sw + j * PW;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (ok[k]) {
                        T in = T(0);
#pragma unroll
                        for (int a = 0; a < W2; ++a) in = fma(wp[a], H[k][a], in);
                        sum = fma(wp[W2 + bb[k]] * wp[2 * W2 + cc[k]], in, sum);
                    }
                }
            }
            part[j] = sum;
        }
        // reduce-scatter over the warp: afterwards lane j holds the warp's sum
        // for point j of the chunk
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const bool upper = lane & o;
#pragma unroll
            for (int kk = 0; kk < o; ++kk) {
                T send = upper ? part[kk] : part[kk + o];
                T keep = upper ? part[kk + o] : part[kk];
                part[kk] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        T tot = part[0];
        if (NW > 1) {
            if (warp == 0) sred[lane] = tot;
            __syncthreads();
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                if (warp == w) sred[lane] += tot;
                __syncthreads();
            }
            tot = sred[lane];
        }
        if (warp == 0 && lane < cn) Y[(int64_t)l * N + perm[start + c0 + lane]] = (double)tot;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ grid convolution
// One CTA = 16 grid lines along `axis`, staged through shared memory so that
// global loads and stores are contiguous rows.  Each warp takes two real
// lines as one complex line of length n = 32 R (element e at lane e % 32,
// register e / 32), runs a radix-2 decimation-in-frequency FFT (output in
// bit-reversed order), multiplies by the bit-reversed multiplier table, and
// runs the decimation-in-time inverse FFT (bit-reversed in, natural out).
// Because the multiplier is real and even, the real and imaginary parts stay
// the two independent convolved lines.
template <typename T, int R>
__global__ void __launch_bounds__(256)
k_conv(T *__restrict__ grid, int axis, const T *__restrict__ tab,
       const typename Vec2<T>::type *__restrict__ tw, const int *__restrict__ done) {
    using C = typename Vec2<T>::type;
    constexpr int n = 32 * R, LPC = 16, PITCH = n + 1;
    __shared__ T S[LPC * PITCH];
    if (done && *done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T *g = grid + (int64_t)blockIdx.y * n * n * n;
    const int li0 = blockIdx.x * LPC;  // first line of the CTA
    const int a0 = li0 % n, b0 = li0 / n;
    // element (line j, position e) -> global offset
    auto goff = [&](int j, int e) -> int64_t {
        if (axis == 0) return ((int64_t)b0 * n + a0 + j) * n + e;          // lines (y, z)
        if (axis == 1) return (int64_t)b0 * n * n + (int64_t)e * n + a0 + j;  // lines (x, z)
        return (int64_t)e * n * n + (int64_t)b0 * n + a0 + j;                 // lines (x, y)
    };
    if (axis == 0) {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q / n, e = q % n;
            S[j * PITCH + e] = g[goff(j, e)];
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            S[j * PITCH + e] = g[goff(j, e)];
        }
    }
    __syncthreads();

    C x[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
        x[r] = {S[(2 * warp) * PITCH + 32 * r + lane], S[(2 * warp + 1) * PITCH + 32 * r + lane]};
    // forward DIF
#pragma unroll
    for (int h = n / 2; h >= 32; h >>= 1) {
        const int H = h / 32;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & H) == 0) {
                C a = x[r], b = x[r + H];
                x[r] = cadd(a, b);
                int j = ((r % H) * 32 + lane) * (n / (2 * h));
                x[r + H] = cmul(csub(a, b), tw[j]);
            }
        }
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const C w = tw[(lane & (h - 1)) * (n / (2 * h))];
        const bool upper = lane & h;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C o = cshfl(x[r], h);
            x[r] = upper ? cmul(csub(o, x[r]), w) : cadd(x[r], o);
        }
    }
    // multiply (table is in bit-reversed order, like the data)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        T f = tab[32 * r + lane];
        x[r].x *= f;
        x[r].y *= f;
    }
    // inverse DIT
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1) {
        const C w = tw[(lane & (h - 1)) * (n / (2 * h))];
        const bool upper = lane & h;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C mine = upper ? cmulc(x[r], w) : x[r];
            C o = cshfl(mine, h);
            x[r] = upper ? csub(o, mine) : cadd(mine, o);
        }
    }
#pragma unroll
    for (int h = 32; h <= n / 2; h <<= 1) {
        const int H = h / 32;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & H) == 0) {
                int j = ((r % H) * 32 + lane) * (n / (2 * h));
                C b = cmulc(x[r + H], tw[j]);
                C a = x[r];
                x[r] = cadd(a, b);
                x[r + H] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        S[(2 * warp) * PITCH + 32 * r + lane] = x[r].x;
        S[(2 * warp + 1) * PITCH + 32 * r + lane] = x[r].y;
    }
    __syncthreads();
    if (axis == 0) {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q / n, e = q % n;
            g[goff(j, e)] = S[j * PITCH + e];
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            g[goff(j, e)] = S[j * PITCH + e];
        }
    }
}

// ------------------------------------------------------------------ epilogue
// y = (1/L) sum_l Y_l; op 1: d o x - y; op 2: alpha x + d o x - y.
// Also clears the grids for the next matvec and writes per-block partial
// sums of x^T y (if partials != NULL).
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_epilogue(const double *__restrict__ Y, int L, int64_t N, const double *__restrict__ x,
           const double *__restrict__ d, double alpha, int op, double *__restrict__ y,
           double *__restrict__ partials, T *__restrict__ grid, int64_t grid_elems,
           const int *__restrict__ done) {
    __shared__ double sh[33];
    if (done && *done) return;
    const double invL = 1.0 / L;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s += Y[(int64_t)l * N + i];
        s *= invL;
        double out;
        if (op == 0) {
            out = s;
        } else {
            double xi = x[i];
            out = d[i] * xi - s;
            if (op == 2) out = fma(alpha, xi, out);
        }
        y[i] = out;
        if (partials) acc = fma(x[i], out, acc);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < grid_elems; i += stride)
        grid[i] = T(0);
    if (partials) {
        double bs = block_sum(acc, sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    }
}

// ------------------------------------------------------------------ dispatch
template <typename T, int W2>
static void launch_spread_interp(Plan &P, bool spread, const T *wts, T *grid,
                                 const double *v, const int *done, cudaStream_t s) {
    constexpr int NW = W2 <= 8 ? 1 : 2;
    if (P.n_items == 0) return;
    if (spread)
        k_spread<T, W2, NW><<<(unsigned)P.n_items, 32 * NW, 0, s>>>(P.items, P.perm, wts, v,
                                                                    grid, P.n, P.m, done);
    else
        k_interp<T, W2, NW><<<(unsigned)P.n_items, 32 * NW, 0, s>>>(P.items, P.perm, wts, grid,
                                                                    P.Y, P.n, P.m, P.N, done);
    NLH_CHECK_LAUNCH();
}

template <typename T>
static void spread_interp(Plan &P, bool spread, const T *wts, T *grid, const double *v,
                          const int *done, cudaStream_t s) {
    switch (P.W2) {
        case 4: launch_spread_interp<T, 4>(P, spread, wts, grid, v, done, s); break;
        case 6: launch_spread_interp<T, 6>(P, spread, wts, grid, v, done, s); break;
        case 8: launch_spread_interp<T, 8>(P, spread, wts, grid, v, done, s); break;
        case 10: launch_spread_interp<T, 10>(P, spread, wts, grid, v, done, s); break;
        case 12: launch_spread_interp<T, 12>(P, spread, wts, grid, v, done, s); break;
        case 14: launch_spread_interp<T, 14>(P, spread, wts, grid, v, done, s); break;
        case 16: launch_spread_interp<T, 16>(P, spread, wts, grid, v, done, s); break;
        default: NLH_REQUIRE(false, "internal: unsupported stencil width %d", P.W2);
    }
}

template <typename T>
static void convolve(Plan &P, T *grid, const T *tab, const typename Vec2<T>::type *tw,
                     const int *done, cudaStream_t s) {
    const int n = P.n;
    dim3 gdim((unsigned)(n * n / 16), (unsigned)P.L);
    for (int axis = 0; axis < 3; ++axis) {
        switch (n) {
            case 32: k_conv<T, 1><<<gdim, 256, 0, s>>>(grid, axis, tab, tw, done); break;
            case 64: k_conv<T, 2><<<gdim, 256, 0, s>>>(grid, axis, tab, tw, done); break;
            case 128: k_conv<T, 4><<<gdim, 256, 0, s>>>(grid, axis, tab, tw, done); break;
            case 256: k_conv<T, 8><<<gdim, 256, 0, s>>>(grid, axis, tab, tw, done); break;
            default: NLH_REQUIRE(false, "internal: unsupported grid size %d", n);
        }
        NLH_CHECK_LAUNCH();
    }
}

template <typename T>
static void matvec_t(Plan &P, int op, double alpha, const double *x, double *y,
                     double *partials, const int *done, const T *wts, T *grid, const T *tab,
                     const typename Vec2<T>::type *tw, const double *d, cudaStream_t s) {
    spread_interp<T>(P, true, wts, grid, x, done, s);
    convolve<T>(P, grid, tab, tw, done, s);
    spread_interp<T>(P, false, wts, grid, nullptr, done, s);
    const int64_t ge = (int64_t)P.L * P.n * P.n * P.n;
    k_epilogue<T><<<kRedBlocks, kRedThreads, 0, s>>>(P.Y, P.L, P.N, x, d, alpha, op, y, partials,
                                                     grid, ge, done);
    NLH_CHECK_LAUNCH();
}

void matvec(Plan &P, int op, int prec, double alpha, const double *x, double *y,
            double *partials, const int *done, cudaStream_t s) {
    if (prec == NLH_FP64) {
        NLH_REQUIRE(P.precision & 1, "matvec: FP64 path not built in this plan");
        matvec_t<double>(P, op, alpha, x, y, partials, done, P.wts64, P.grid64, P.tab64, P.tw64,
                         P.d64, s);
    } else {
        NLH_REQUIRE(P.precision & 2, "matvec: FP32 path not built in this plan");
        matvec_t<float>(P, op, alpha, x, y, partials, done, P.wts32, P.grid32, P.tab32, P.tw32,
                        P.d32, s);
    }
}

}  // namespace nlh

extern "C" nlh_status nlh_matvec(nlh_plan plan, int op, int precision, double alpha,
                                 const double *x, double *y, void *stream) {
    nlh::clear_error();
    try {
        NLH_REQUIRE(plan && x && y, "nlh_matvec: NULL pointer");
        NLH_REQUIRE(x != y, "nlh_matvec: x and y must not alias");
        NLH_REQUIRE(op >= 0 && op <= 2, "nlh_matvec: op=%d", op);
        NLH_REQUIRE(precision == NLH_FP64 || precision == NLH_FP32, "nlh_matvec: precision=%d",
                    precision);
        nlh::matvec(*plan, op, precision, alpha, x, y, nullptr, nullptr, (cudaStream_t)stream);
        return NLH_OK;
    } catch (nlh::Failure &f) {
        return f.st;
    }
}
