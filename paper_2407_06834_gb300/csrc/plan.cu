// plan.cu -- plan construction: features, torus map, sort by grid cell,
// work items, window weights and Fourier multiplier tables.
//
// Paper: arXiv 2407.06834.  Patches and windows: Sec. 5.  Fast summation
// per window (adjoint NFFT, multiply by the Gaussian's Fourier coefficients,
// NFFT): Sec. 3, Eq. NFFT and Eq. DGT.  Degrees eta = Gamma 1: Sec. 2.3.
#include "common.cuh"
#include "df32.cuh"

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

namespace nlh {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }

// Pinned host mirrors and capture streams cost a driver round trip (page
// pinning, stream creation) that a plan made per image would pay every
// time; plans take them from process-wide free lists and return them.
namespace {
struct HostPool {
    std::mutex mu;
    std::vector<SolveState *> st;
    std::vector<double *> red;
    std::map<int, std::vector<cudaStream_t>> streams;  // per device
};
HostPool &host_pool() {
    static HostPool *p = new HostPool();  // kept to process exit
    return *p;
}
}  // namespace

void take_pinned(Plan &P) {
    HostPool &hp = host_pool();
    {
        std::lock_guard<std::mutex> lk(hp.mu);
        if (!hp.st.empty()) { P.st_host = hp.st.back(); hp.st.pop_back(); }
        if (!hp.red.empty()) { P.red_host = hp.red.back(); hp.red.pop_back(); }
    }
    if (!P.st_host) NLH_CUDA(cudaMallocHost(&P.st_host, sizeof(SolveState)));
    if (!P.red_host) NLH_CUDA(cudaMallocHost(&P.red_host, sizeof(double) * 3 * kRedBlocks));
}

cudaStream_t take_capture_stream(int device) {
    HostPool &hp = host_pool();
    {
        std::lock_guard<std::mutex> lk(hp.mu);
        auto &v = hp.streams[device];
        if (!v.empty()) {
            cudaStream_t s = v.back();
            v.pop_back();
            return s;
        }
    }
    cudaStream_t s = nullptr;
    NLH_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    return s;
}

void give_capture_stream(int device, cudaStream_t s) {
    HostPool &hp = host_pool();
    std::lock_guard<std::mutex> lk(hp.mu);
    hp.streams[device].push_back(s);
}

Plan::~Plan() {
    cudaStreamSynchronize(stream);
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    for (void *ptr : allocs) cudaFreeAsync(ptr, stream);
    HostPool &hp = host_pool();
    std::lock_guard<std::mutex> lk(hp.mu);
    if (st_host) hp.st.push_back(st_host);
    if (red_host) hp.red.push_back(red_host);
    if (capture_stream) hp.streams[device].push_back(capture_stream);
}

// Destroy the plan's cached solve graphs (they hold the work-item and unit
// arrays and the kernels' launch shapes); the next solve captures afresh.
void drop_graphs(Plan &P) {
    ++P.graph_epoch;  // batch graphs that hold this plan's solve are stale too
    if (P.graphs.empty()) return;
    NLH_CUDA(cudaStreamSynchronize(P.stream));
    for (auto &kv : P.graphs) cudaGraphExecDestroy(kv.second);
    P.graphs.clear();
}

void retain_pool_memory() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// ------------------------------------------------------------------ features

// Patch features (Sec. 5): one thread per (pixel, patch dim).
__global__ void k_patch_features(const double *__restrict__ img, int n1, int n2,
                                 int rho, int pad, double *__restrict__ feat) {
    const int P = 2 * rho + 1, D = P * P;
    const int64_t total = (int64_t)n1 * n2 * D;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t pix = idx / D;
        int k = (int)(idx - pix * D);
        int r = (int)(pix / n2), c = (int)(pix - (int64_t)r * n2);
        int rr = r + k / P - rho, cc = c + k % P - rho;
        double val;
        if (pad == 0) {
            val = (rr < 0 || rr >= n1 || cc < 0 || cc >= n2) ? 0.0 : img[(int64_t)rr * n2 + cc];
        } else {
            val = img[(int64_t)reflect_index(rr, n1) * n2 + reflect_index(cc, n2)];
        }
        feat[idx] = val;
    }
}

__device__ __forceinline__ double window_coord(const double *__restrict__ feat, int D,
                                               const int *__restrict__ win, int l,
                                               int64_t i, int t) {
    int d = win[3 * l + t];
    return d < 0 ? 0.0 : feat[i * D + d];
}

// ------------------------------------------------------------------ min/max
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// blockIdx.y = coordinate (window l, dim t); partial min / max per block.
__global__ void k_minmax_partial(const double *__restrict__ feat, int64_t N, int D,
                                 const int *__restrict__ win, double *__restrict__ part) {
    __shared__ double smin[32], smax[32];
    int coord = blockIdx.y, l = coord / 3, t = coord % 3;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = window_coord(feat, D, win, l, i, t);
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { smin[wid] = lo; smax[wid] = hi; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        lo = lane < nw ? smin[lane] : INFINITY;
        hi = lane < nw ? smax[lane] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            part[((int64_t)coord * gridDim.x + blockIdx.x) * 2 + 0] = lo;
            part[((int64_t)coord * gridDim.x + blockIdx.x) * 2 + 1] = hi;
        }
    }
}

__global__ void k_minmax_final(const double *__restrict__ part, int nb, double *__restrict__ mm) {
    int coord = blockIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    for (int j = threadIdx.x; j < nb; j += 32) {
        lo = fmin(lo, part[((int64_t)coord * nb + j) * 2 + 0]);
        hi = fmax(hi, part[((int64_t)coord * nb + j) * 2 + 1]);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (threadIdx.x == 0) { mm[2 * coord] = lo; mm[2 * coord + 1] = hi; }
}

// ------------------------------------------------------------------ sort by cell
// Cells are ordered tile-major: tiles of kTile^3 cells in (z, y, x) order,
// then the cells inside a tile in (z, y, x) order.  The map is a bijection
// of [0, n^3), so a counting sort over it groups the points of each cell and
// keeps the cells of one tile contiguous.
__device__ __forceinline__ int tile_major_key(int x, int y, int z, int n) {
    const int nt = n / kTile;
    int tile = ((z / kTile) * nt + y / kTile) * nt + x / kTile;
    int local = ((z % kTile) * kTile + y % kTile) * kTile + x % kTile;
    return tile * (kTile * kTile * kTile) + local;
}

// Grid coordinate u = (s (x - c) + 1/2) n taken modulo n, so that the torus
// [-1/2, 1/2) maps to the grid points 0..n-1.  Cell = floor(u).
__global__ void k_cell_keys(const double *__restrict__ feat, int64_t N, int D, int L,
                            const int *__restrict__ win, const double *__restrict__ center,
                            double s, int n, double *__restrict__ u, int *__restrict__ keys,
                            int *__restrict__ hist) {
    const int64_t total = (int64_t)L * N;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int l = (int)(idx / N);
        int64_t i = idx - (int64_t)l * N;
        int cell[3];
        for (int t = 0; t < 3; ++t) {
            double x = window_coord(feat, D, win, l, i, t);
            double ut = (s * (x - center[3 * l + t]) + 0.5) * n;
            ut -= n * floor(ut / n);
            if (ut >= n) ut -= n;
            if (ut < 0.0) ut = 0.0;
            int c = (int)floor(ut);
            if (c > n - 1) c = n - 1;
            u[idx * 3 + t] = ut;
            cell[t] = c;
        }
        int key = tile_major_key(cell[0], cell[1], cell[2], n);
        keys[idx] = key;
        atomicAdd(&hist[(int64_t)l * n3 + key], 1);
    }
}

__global__ void k_scatter(const int *__restrict__ keys, int64_t N, int L, int64_t n3,
                          int *__restrict__ cursor, int *__restrict__ perm) {
    const int64_t total = (int64_t)L * N;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int l = (int)(idx / N);
        int64_t i = idx - (int64_t)l * N;
        int pos = atomicAdd(&cursor[(int64_t)l * n3 + keys[idx]], 1);
        perm[pos] = (int)i;
    }
}

// ------------------------------------------------------------------ exclusive scan (int32)
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int block_incl_scan(int v, int *sh /* 32 */) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += sh[wid - 1];
    __syncthreads();
    return v;
}

__global__ void k_scan_tiles(const int *__restrict__ in, int64_t n, int *__restrict__ sums) {
    __shared__ int sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int v = 0;
    for (int j = 0; j < kScanPer; ++j)
        if (base + j < n) v += in[base + j];
    v = block_incl_scan(v, sh);
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = v;
}

__global__ void k_scan_sums(int *__restrict__ sums, int nt, int *__restrict__ total) {
    __shared__ int sh[32];
    __shared__ int last;
    int carry = 0;
    for (int base = 0; base < nt; base += kScanThreads) {
        int i = base + threadIdx.x;
        int v = i < nt ? sums[i] : 0;
        int inc = block_incl_scan(v, sh);
        if (i < nt) sums[i] = carry + inc - v;
        if (threadIdx.x == kScanThreads - 1) last = inc;
        __syncthreads();
        carry += last;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int *__restrict__ in, int64_t n, const int *__restrict__ sums,
                             int *__restrict__ out) {
    __shared__ int sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int vals[kScanPer];
    int v = 0;
    for (int j = 0; j < kScanPer; ++j) {
        vals[j] = (base + j < n) ? in[base + j] : 0;
        v += vals[j];
    }
    int inc = block_incl_scan(v, sh);
    int run = sums[blockIdx.x] + inc - v;
    for (int j = 0; j < kScanPer; ++j) {
        if (base + j < n) out[base + j] = run;
        run += vals[j];
    }
}

// out = exclusive scan of in, the total to d_total, no synchronisation.
static void exclusive_scan_dev(const int *in, int *out, int64_t n, cudaStream_t s,
                               int *tmp_sums, int *d_total) {
    int nt = div_up(n, kScanTile);
    k_scan_tiles<<<nt, kScanThreads, 0, s>>>(in, n, tmp_sums);
    NLH_CHECK_LAUNCH();
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp_sums, nt, d_total);
    NLH_CHECK_LAUNCH();
    k_scan_apply<<<nt, kScanThreads, 0, s>>>(in, n, tmp_sums, out);
    NLH_CHECK_LAUNCH();
}

// out = exclusive scan of in; returns the total (synchronises s).
static int64_t exclusive_scan(Plan &P, const int *in, int *out, int64_t n, cudaStream_t s,
                              int *tmp_sums, int *d_total) {
    int nt = div_up(n, kScanTile);
    k_scan_tiles<<<nt, kScanThreads, 0, s>>>(in, n, tmp_sums);
    NLH_CHECK_LAUNCH();
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp_sums, nt, d_total);
    NLH_CHECK_LAUNCH();
    k_scan_apply<<<nt, kScanThreads, 0, s>>>(in, n, tmp_sums, out);
    NLH_CHECK_LAUNCH();
    int total = 0;
    NLH_CUDA(cudaMemcpyAsync(&total, d_total, sizeof(int), cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    return total;
}

// ------------------------------------------------------------------ work items
__global__ void k_item_counts(const int *__restrict__ hist, int64_t ncells, int kmax,
                              int *__restrict__ cnt, int *__restrict__ occupied) {
    int occ = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int h = hist[c];
        cnt[c] = (h + kmax - 1) / kmax;
        occ += h > 0;
    }
    occ = __reduce_add_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && occ) atomicAdd(occupied, occ);
}

__global__ void k_emit_items(const int *__restrict__ hist, const int *__restrict__ start,
                             const int *__restrict__ item_off, int64_t ncells, int n,
                             int kmax, int4 *__restrict__ items) {
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int h = hist[c];
        if (h == 0) continue;
        int l = (int)(c / n3);
        const int key = (int)(c - (int64_t)l * n3), t3 = kTile * kTile * kTile;
        const int tile = key / t3, local = key % t3;  // tile-major key
        const int lx = local % kTile, ly = (local / kTile) % kTile, lz = local / (kTile * kTile);
        const int packed = (l << 16) | (lz << 6) | (ly << 3) | lx;
        int o = item_off[c];
        for (int t = 0; t * kmax < h; ++t)
            items[o + t] = make_int4(packed, tile, start[c] + t * kmax, min(kmax, h - t * kmax));
    }
}

// ------------------------------------------------------------------ window weights
// Kaiser-Bessel window (Kaiser 1974; its use for gridding: Jackson et al.
// 1991): phi(x) = I0(beta sqrt(1 - (n x / m)^2)) / I0(beta) for |n x| <= m.
// A point at grid coordinate u = c + f (c integer, 0 <= f < 1) touches the
// 2m grid points g = c - m + 1 + j, j = 0..2m-1, at offsets g - u in
// (-m, m], with weight P_j(f) = phi((j - m + 1 - f) / m).  Because
// I0(beta sqrt(z)) is an entire function of z, each P_j is analytic on
// [0, 1].  With y = 2 f - 1, P_{2m-1-j}(y) = P_j(-y), so only j < m is
// fitted: Chebyshev interpolation of P_j in y of a fixed degree, converted to
// monomials and split into the even part E_j(y^2) and the odd part
// y O_j(y^2) (window.cuh evaluates both weights of a pair from them).  The
// fit is checked on the host against direct Bessel evaluation, for both
// weights of every pair.
static double kb_host(double x, double beta) {
    double z = 1.0 - x * x;
    if (z < 0.0) return 0.0;
    return std::cyl_bessel_i(0.0, beta * std::sqrt(z)) / std::cyl_bessel_i(0.0, beta);
}

// Monomial coefficients a[j][k], k < K, of the degree-(K-1) Chebyshev
// interpolant of P_j, j < m; returns the largest deviation from the window
// over both weights of each pair on a fine grid of y.
static double fit_pairs(int m, double beta, int K, std::vector<double> &a) {
    a.assign((size_t)m * K, 0.0);
    double worst = 0.0;
    for (int j = 0; j < m; ++j) {
        auto Pj = [&](double y) { return kb_host((j - m + 1 - 0.5 * (y + 1.0)) / m, beta); };
        std::vector<double> c(K, 0.0), g(K);
        for (int i = 0; i < K; ++i) g[i] = Pj(std::cos(M_PI * (i + 0.5) / K));
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int i = 0; i < K; ++i) acc += g[i] * std::cos(M_PI * k * (i + 0.5) / K);
            c[k] = (k == 0 ? 1.0 : 2.0) * acc / K;
        }
        // Chebyshev -> monomial: T_{k+1} = 2 y T_k - T_{k-1}
        std::vector<double> tkm1(K, 0.0), tk(K, 0.0), mono(K, 0.0);
        tkm1[0] = 1.0;
        if (K > 1) tk[1] = 1.0;
        for (int i = 0; i < K; ++i) mono[i] += c[0] * tkm1[i];
        if (K > 1)
            for (int i = 0; i < K; ++i) mono[i] += c[1] * tk[i];
        for (int k = 2; k < K; ++k) {
            std::vector<double> tn(K, 0.0);
            for (int i = 0; i < K; ++i) {
                if (i > 0) tn[i] += 2.0 * tk[i - 1];
                tn[i] -= tkm1[i];
            }
            for (int i = 0; i < K; ++i) mono[i] += c[k] * tn[i];
            tkm1 = tk;
            tk = tn;
        }
        for (int i = 0; i < K; ++i) a[(size_t)j * K + i] = mono[i];
        const int jm = 2 * m - 1 - j;
        for (int q = 0; q <= 400; ++q) {
            const double y = -1.0 + q / 200.0, u = y * y;
            double e = 0.0, o = 0.0;
            for (int k = (K - 1) / 2 * 2; k >= 0; k -= 2) e = e * u + mono[k];
            for (int k = (K - 2) / 2 * 2 + 1; k >= 1; k -= 2) o = o * u + mono[k];
            const double fx = (jm - m + 1 - 0.5 * (y + 1.0)) / m;
            worst = std::max(worst, std::fabs(e + y * o - Pj(y)));
            worst = std::max(worst, std::fabs(e - y * o - kb_host(fx, beta)));
        }
    }
    return worst;
}

// The three coefficient sets of a plan (cached per (m, beta): they depend on
// nothing else).  FP64 and double-float: degree 15, <= 2e-14 off the window;
// FP32: degree 9, <= 1e-7 (below what FP32 weights resolve).
struct WinSets {
    WinPoly<float> f32;
    WinPoly<double> f64;
    WinPoly<df32> fdf;
};

static WinSets fit_window(int m, double beta) {
    static std::mutex mu;
    static std::map<std::pair<int, double>, WinSets> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(m, beta);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    NLH_REQUIRE(m >= 1 && m <= kWinHalfMax, "internal: window half-width %d", m);
    WinSets w;
    std::memset(&w, 0, sizeof w);
    std::vector<double> a64, a32;
    const double e64 = fit_pairs(m, beta, 2 * kWinK64, a64);
    const double e32 = fit_pairs(m, beta, 2 * kWinK32, a32);
    NLH_REQUIRE(e64 <= 2e-14 && e32 <= 1e-7,
                "window polynomials do not reach their accuracy for m=%d, beta=%g (%.2e, %.2e)", m,
                beta, e64, e32);
    for (int j = 0; j < m; ++j)
        for (int par = 0; par < 2; ++par) {
            for (int k = 0; k < kWinK64; ++k) {
                const double c = a64[(size_t)j * 2 * kWinK64 + 2 * k + par];
                w.f64.c[j][par][k] = c;
                const float hi = (float)c;
                w.fdf.hi[j][par][k] = hi;
                w.fdf.lo[j][par][k] = (float)(c - (double)hi);
            }
            for (int k = 0; k < kWinK32; ++k)
                w.f32.c[j][par][k] = (float)a32[(size_t)j * 2 * kWinK32 + 2 * k + par];
        }
    cache.emplace(key, w);
    return w;
}

// (hi, lo) float pair of each pixel value (FP32 path of a plan that
// recomputes coordinates from the image).
__global__ void k_split_image(const double *__restrict__ img, int64_t N,
                              float2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = img[i];
        const float hi = (float)v;
        out[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

// Cell offsets of the sorted points: y = 2 (u - floor u) - 1 per dim (u the
// grid coordinate of k_cell_keys), as a float and the float remainder.
__global__ void k_offsets(const int *__restrict__ perm, const double *__restrict__ u, int64_t N,
                          int L, float *__restrict__ yhi, float *__restrict__ ylo) {
    const int64_t total = (int64_t)L * N;
    for (int64_t sidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sidx < total;
         sidx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(sidx / N);
        const int64_t i = perm[sidx];
        const double *up = u + ((int64_t)l * N + i) * 3;
        for (int t = 0; t < 3; ++t) {
            const double ut = up[t];
            const double y = 2.0 * (ut - floor(ut)) - 1.0;
            const float hi = (float)y;
            yhi[sidx * 3 + t] = hi;
            if (ylo) ylo[sidx * 3 + t] = (float)(y - (double)hi);
        }
    }
}

// ------------------------------------------------------------------ multiplier tables
// Per dim, the adjoint NFFT, the multiply by the Gaussian's Fourier
// coefficients and the NFFT (Sec. 3) collapse into one circular convolution
// of the oversampled grid with the real, even multiplier
//   w(k) = 1_{|k| < M/2} ghat(k) / (n chat(k))^2,
//   ghat(k) = sqrt(pi) sigma_s exp(-pi^2 sigma_s^2 k^2)  (Gaussian transform),
//   chat(k) = (2m/n) sinh(z)/z / I0(beta), z = sqrt(beta^2 - (2 pi m k/n)^2)
// (transform of the Kaiser-Bessel window above).  The table is stored in
// bit-reversed order for the FFT of nfft.cu.
__global__ void k_tables(int n, int logn, int M, int m, double beta, double inv_i0b,
                         double sigma_s, double *__restrict__ tab64, float *__restrict__ tab32,
                         double2 *__restrict__ tw64, float2 *__restrict__ tw32,
                         float2 *__restrict__ tabdf, float4 *__restrict__ twdf) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int kk = (int)(__brev((unsigned)j) >> (32 - logn));
    int f = kk < n / 2 ? kk : kk - n;
    double w = 0.0;
    if (2 * abs(f) < M) {
        const double pi = 3.141592653589793238462643;
        double om = 2.0 * pi * m * f / n;
        double z2 = beta * beta - om * om;
        double shz;
        if (z2 > 1e-24) {
            double z = sqrt(z2);
            shz = sinh(z) / z;
        } else {
            shz = 1.0;
        }
        double chat = (2.0 * m / n) * shz * inv_i0b;
        double ghat = sqrt(pi) * sigma_s * exp(-pi * pi * sigma_s * sigma_s * (double)f * f);
        double nc = n * chat;
        w = ghat / (nc * nc);
    }
    if (tab64) tab64[j] = w;
    if (tab32) tab32[j] = (float)w;
    if (tabdf) tabdf[j] = make_float2((float)w, (float)(w - (double)(float)w));
    if (j < n / 2) {
        double sn, cs;
        sincospi(2.0 * j / n, &sn, &cs);
        if (tw64) tw64[j] = make_double2(cs, -sn);
        if (tw32) tw32[j] = make_float2((float)cs, (float)-sn);
        if (twdf)
            twdf[j] = make_float4((float)cs, (float)(cs - (double)(float)cs), (float)-sn,
                                  (float)(-sn - (double)(float)-sn));
    }
}

__global__ void k_fill(double *__restrict__ x, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// Work units: runs of consecutive items (tile-major order) of one window and
// one tile.  An item belongs to the unit given by the bucket of its point
// offset inside the (window, tile) group (unit_points points per bucket) and
// of its item index inside the group (kUnitItems per bucket); a unit may
// exceed unit_points by its last item.  Units are then ordered by
// decreasing point count so that the largest start first (a counting sort
// on the size; the order among units of one size is not fixed).  All on the
// device, in data-parallel passes: the unit count stays in device memory
// (P.d_units[0]) for the persistent kernels and reaches the host at the
// plan's next synchronisation.
constexpr int kSizeBins = 4096;

// (window, tile) group of an item; ntiles = tiles per window
__device__ __forceinline__ int group_key(const int4 &it, int ntiles) {
    return (it.x >> 16) * ntiles + it.y;
}

// pts[i] = point count of item i; first[g] = min item index of group g.
__global__ void k_item_pts(const int4 *__restrict__ items, int64_t n_items, int ntiles,
                           int *__restrict__ pts, int *__restrict__ first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int4 it = items[i];
        pts[i] = it.w;
        if (i == 0 || group_key(items[i - 1], ntiles) != group_key(it, ntiles))
            first[group_key(it, ntiles)] = (int)i;
    }
}

// brk[i] = 1 where item i starts a unit (a new group, or a new point or item
// bucket inside the group).
__device__ __forceinline__ long long unit_bucket(int64_t i, const int4 *items, const int *pre,
                                                 const int *first, int ntiles, int unit_points) {
    const int g0 = first[group_key(items[i], ntiles)];
    const long long pb = (pre[i] - pre[g0]) / unit_points;
    const long long ib = (i - g0) / kUnitItems;
    return pb * 1048576ll + ib;
}

__global__ void k_unit_breaks(const int4 *__restrict__ items, int64_t n_items, int ntiles,
                              const int *__restrict__ pre, const int *__restrict__ first,
                              int unit_points, int *__restrict__ brk) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x) {
        int b = 1;
        if (i > 0 && group_key(items[i - 1], ntiles) == group_key(items[i], ntiles))
            b = unit_bucket(i - 1, items, pre, first, ntiles, unit_points) !=
                unit_bucket(i, items, pre, first, ntiles, unit_points);
        brk[i] = b;
    }
}

// start[uid[i]] = i at each unit start (uid = exclusive scan of brk).
__global__ void k_unit_starts(const int *__restrict__ brk, const int *__restrict__ uid,
                              int64_t n_items, int *__restrict__ start) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x)
        if (brk[i]) start[uid[i]] = (int)i;
}

// Unit u covers items start[u] .. start[u+1]-1 (or to the end).
__global__ void k_unit_emit(const int4 *__restrict__ items, int64_t n_items,
                            const int *__restrict__ start, const int *__restrict__ pre,
                            const int *__restrict__ n_units, int4 *__restrict__ units,
                            int *__restrict__ sizes) {
    const int nu = *n_units;
    const int total = pre[n_items - 1] + items[n_items - 1].w;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
        const int i0 = start[u];
        const int i1 = u + 1 < nu ? start[u + 1] : (int)n_items;
        units[u] = make_int4(items[i0].x >> 16, items[i0].y, i0, i1 - i0);
        sizes[u] = (i1 < n_items ? pre[i1] : total) - pre[i0];
    }
}

__global__ void k_size_hist(const int *__restrict__ sizes, const int *__restrict__ n_units,
                            int *__restrict__ hist) {
    const int n = *n_units;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&hist[min(sizes[i], kSizeBins - 1)], 1);
}

// off[b] = number of units in bins above b (descending order of size).
__global__ void k_size_offsets(const int *__restrict__ hist, int *__restrict__ off) {
    __shared__ int sh[32];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < kSizeBins; base += blockDim.x) {
        const int b = kSizeBins - 1 - (base + (int)threadIdx.x);  // descending
        const int v = hist[b];
        const int inc = block_incl_scan(v, sh);
        off[b] = carry_s + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s += inc;
        __syncthreads();
    }
}

__global__ void k_size_scatter(const int4 *__restrict__ in, const int *__restrict__ sizes,
                               const int *__restrict__ n_units, int *__restrict__ off,
                               int4 *__restrict__ out) {
    const int n = *n_units;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[atomicAdd(&off[min(sizes[i], kSizeBins - 1)], 1)] = in[i];
}

static void exclusive_scan_dev(const int *in, int *out, int64_t n, cudaStream_t s,
                               int *tmp_sums, int *d_total);

static void build_units(Plan &P, cudaStream_t s) {
    const int64_t ni = P.n_items;
    if (P.units) P.release(P.units);
    P.units = P.alloc<int4>(std::max<int64_t>(ni, 1));
    P.units_cap = ni;
    if (!P.d_units) P.d_units = P.alloc<int>(1);
    NLH_CUDA(cudaMemsetAsync(P.d_units, 0, sizeof(int), s));
    if (ni == 0) return;
    const int nt = P.n / kTile, nt3 = nt * nt * nt;
    const int64_t ngroups = (int64_t)P.L * nt3;
    int *pts = nullptr, *pre = nullptr, *first = nullptr, *brk = nullptr, *uid = nullptr,
        *sums = nullptr, *sizes = nullptr, *hist = nullptr, *off = nullptr, *tot = nullptr,
        *start = nullptr;
    int4 *tmpu = nullptr;
    std::vector<void *> tmp;
    auto talloc = [&](auto **ptr, size_t bytes) {
        NLH_CUDA(cudaMallocAsync((void **)ptr, std::max<size_t>(bytes, 4), s));
        tmp.push_back(*ptr);
    };
    try {
        talloc(&pts, sizeof(int) * ni);
        talloc(&pre, sizeof(int) * ni);
        talloc(&first, sizeof(int) * ngroups);
        talloc(&brk, sizeof(int) * ni);
        talloc(&uid, sizeof(int) * ni);
        talloc(&start, sizeof(int) * ni);
        talloc(&sums, sizeof(int) * (div_up(ni, kScanTile) + 1));
        talloc(&sizes, sizeof(int) * ni);
        talloc(&tmpu, sizeof(int4) * ni);
        talloc(&hist, sizeof(int) * kSizeBins);
        talloc(&off, sizeof(int) * kSizeBins);
        talloc(&tot, sizeof(int));
        const int gb = (int)std::min<int64_t>(div_up(ni, 256), 152 * 8);
        k_item_pts<<<gb, 256, 0, s>>>(P.items, ni, nt3, pts, first);
        NLH_CHECK_LAUNCH();
        exclusive_scan_dev(pts, pre, ni, s, sums, tot);
        k_unit_breaks<<<gb, 256, 0, s>>>(P.items, ni, nt3, pre, first, P.unit_points, brk);
        NLH_CHECK_LAUNCH();
        exclusive_scan_dev(brk, uid, ni, s, sums, P.d_units);
        k_unit_starts<<<gb, 256, 0, s>>>(brk, uid, ni, start);
        NLH_CHECK_LAUNCH();
        k_unit_emit<<<gb, 256, 0, s>>>(P.items, ni, start, pre, P.d_units, tmpu, sizes);
        NLH_CHECK_LAUNCH();
        NLH_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * kSizeBins, s));
        k_size_hist<<<gb, 256, 0, s>>>(sizes, P.d_units, hist);
        NLH_CHECK_LAUNCH();
        k_size_offsets<<<1, 1024, 0, s>>>(hist, off);
        NLH_CHECK_LAUNCH();
        k_size_scatter<<<gb, 256, 0, s>>>(tmpu, sizes, P.d_units, off, P.units);
        NLH_CHECK_LAUNCH();
    } catch (...) {
        for (void *ptr : tmp) cudaFreeAsync(ptr, s);
        throw;
    }
    for (void *ptr : tmp) cudaFreeAsync(ptr, s);
    P.n_units = -1;  // known on the device; read at the next synchronisation
}

// The host copy of the unit count (after the stream has been synchronised
// or with this call's own synchronisation).
static void fetch_unit_count(Plan &P, cudaStream_t s) {
    int nu = 0;
    if (P.d_units) {
        NLH_CUDA(cudaMemcpyAsync(&nu, P.d_units, sizeof(int), cudaMemcpyDeviceToHost, s));
        NLH_CUDA(cudaStreamSynchronize(s));
    }
    P.n_units = nu;
}

// Re-split the plan's points into items of at most kmax points and units of
// at most unit_points points, in place: the cells of the current items are
// recovered on the host (items of one cell are consecutive and contiguous
// in sorted order) and cut again; no re-sort, no new weights.
static void retile(Plan &P, int kmax, int unit_points, cudaStream_t s) {
    drop_graphs(P);
    std::vector<int4> items(P.n_items);
    if (P.n_items)
        NLH_CUDA(cudaMemcpyAsync(items.data(), P.items, sizeof(int4) * P.n_items,
                                 cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    std::vector<int4> out;
    out.reserve(items.size());
    size_t i = 0;
    while (i < items.size()) {
        int4 cell = items[i];
        size_t j = i + 1;
        while (j < items.size() && items[j].x == cell.x && items[j].y == cell.y &&
               items[j].z == cell.z + cell.w) {
            cell.w += items[j].w;
            ++j;
        }
        for (int t = 0; t < cell.w; t += kmax)
            out.push_back(make_int4(cell.x, cell.y, cell.z + t, std::min(kmax, cell.w - t)));
        i = j;
    }
    if (P.items) P.release(P.items);
    P.n_items = (int64_t)out.size();
    P.items = P.alloc<int4>(out.size());
    if (!out.empty())
        NLH_CUDA(cudaMemcpyAsync(P.items, out.data(), sizeof(int4) * out.size(),
                                 cudaMemcpyHostToDevice, s));
    P.kmax = kmax;
    P.unit_points = unit_points;
    build_units(P, s);
    fetch_unit_count(P, s);
}

static int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// A-priori per-dim error estimates used to pick the torus fill: the Gaussian
// coefficients dropped by the truncation |k| < M/2 sum to at most
// erfc(pi sigma_s (M/2 - 1)); the nearest periodic image of the Gaussian
// sits at distance 1 - fill, giving about 2 exp(-((1 - fill)/sigma_s)^2).
static void error_estimates(double sigma, double R, double fill, int M, double *trunc,
                            double *alias) {
    double ss = sigma * fill / R;
    *trunc = std::erfc(M_PI * ss * (M / 2.0 - 1.0));
    double a = (1.0 - fill) / ss;
    *alias = 2.0 * std::exp(-a * a);
}

// Inverse of erfc on (0, 1] by bisection on std::erfc (monotone).
static double erfc_inv(double y) {
    double lo = 0.0, hi = 10.0;
    for (int k = 0; k < 200; ++k) {
        double mid = 0.5 * (lo + hi);
        if (std::erfc(mid) > y) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// NFFT parameters for a per-dim error target eps (used when nfft_eps > 0):
// alias 2 exp(-((1 - fill)/sigma_s)^2) <= eps gives the torus fill,
// truncation erfc(pi sigma_s (M/2 - 1)) <= eps the bandwidth M, the grid is
// the next power of two >= 2M (oversampling >= 2, at most 256), and the
// Kaiser-Bessel window error ~ exp(-4.44 m) at oversampling 2 gives m.
// NFFT parameters for a per-dim error target eps (nlh_plan_desc.nfft_eps):
// the torus fill and bandwidth M from the alias and truncation bounds, then
// among the grid sizes n_os (powers of two, oversampling n_os / M >= 1.25)
// the one with the least estimated work.  The Kaiser-Bessel window with
// oversampling r = n_os / M has its error decay like
// exp(-2 pi m sqrt(1 - 1/r)) (Sec. 3; for r = 2 that is exp(-4.44 m)), which
// fixes the smallest cutoff m for each n_os; the work of a matvec is about
// N L (2m)^3 stencil updates against L n_os^3 convolved grid cells, whose
// measured relative cost is ~250 updates per cell (x 1.5 for n_os = 256,
// whose axis passes run separately).  Small images (few points per grid
// cell) thus take a smaller grid and a larger cutoff.  Odd cutoffs from 5 up
// are rounded up to the even ones whose stencil widths have tuned kernels.
static void auto_params(double sigma, double R, double eps, int m_in, int64_t NL, int L, int &M,
                        int &n_os, int &m, double &fill) {
    const double a = std::sqrt(std::log(2.0 / eps));
    fill = std::min(0.9, 1.0 / (1.0 + a * sigma / R));
    const double ss = sigma * fill / R;
    const double half = 1.0 + erfc_inv(eps) / (M_PI * ss);
    M = 2 * (int)std::ceil(half);
    if (M < 8) M = 8;
    if (M > 128) M = 128;
    double best = INFINITY;
    n_os = 0;
    m = 0;
    for (int n = 32; n <= 256; n *= 2) {
        const double r = (double)n / M;
        if (r < 1.25) continue;
        int mm = m_in > 0 ? m_in
                          : (int)std::ceil(std::log(1.0 / eps) / (2.0 * M_PI * std::sqrt(1.0 - 1.0 / r)));
        mm = std::min(8, std::max(2, mm));
        if (m_in <= 0 && mm >= 5 && (mm & 1)) ++mm;  // 2m = 12, 16 have the tuned kernel shapes
        if (2 * mm >= n) continue;
        const double w = 2.0 * mm;
        const double cost = (double)NL * w * w * w +
                            250.0 * (n == 256 ? 1.5 : 1.0) * L * (double)n * n * n;
        if (cost < best) {
            best = cost;
            n_os = n;
            m = mm;
        }
    }
    if (n_os == 0) {  // M = 128 with no n_os >= 1.25 M below 256: the largest grid
        n_os = 256;
        m = m_in > 0 ? m_in : std::min(8, std::max(2, (int)std::ceil(std::log(1.0 / eps) / 4.44)));
        if (2 * m >= n_os) m = n_os / 2 - 1;
    }
}

static double choose_fill(double sigma, double R, int M) {
    double best = 0.5, best_err = INFINITY;
    for (int k = 5; k <= 95; ++k) {
        double fill = k / 100.0, tr, al;
        error_estimates(sigma, R, fill, M, &tr, &al);
        double e = std::max(tr, al);
        if (e < best_err) { best_err = e; best = fill; }
    }
    return best;
}

void plan_tables(Plan &P, cudaStream_t s) {
    double sigma_s = P.sigma * P.scale;
    double inv_i0b = 1.0 / std::cyl_bessel_i(0.0, P.kb_beta);
    k_tables<<<div_up(P.n, 256), 256, 0, s>>>(P.n, ilog2(P.n), P.M, P.m, P.kb_beta, inv_i0b,
                                              sigma_s, P.tab64, P.tab32, P.tw64, P.tw32, P.tabdf,
                                              P.twdf);
    NLH_CHECK_LAUNCH();
}

void check_device_error(Plan &P, cudaStream_t s) {
    int e = 0;
    NLH_CUDA(cudaMemcpyAsync(&e, P.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NLH_CUDA(cudaStreamSynchronize(s));
    int chk[5];
    if (nfft_check_take(chk) != 0) {
        set_error("an NFFT kernel found an index of the plan data out of range and skipped it "
                  "(check %d: index %d, bound %d, block %d, thread %d)",
                  chk[0], chk[1], chk[2], chk[3], chk[4]);
        throw Failure{NLH_ERR_CUDA};
    }
    if (e != 0) {
        NLH_CUDA(cudaMemsetAsync(P.err, 0, sizeof(int), s));
        set_error("a bounded device wait did not complete in time (status %d)", e);
        throw Failure{NLH_ERR_TIMEOUT};
    }
}

// d = Gamma_full 1 for each arithmetic of the plan, each from its own
// operator: the deflated methods rely on L 1 = d - Gamma_full 1 = 0 holding
// to the rounding of the arithmetic that applies L.  (Taking the FP32 path's
// degrees from the accurate path leaves L 1 at the FP32 NFFT error times d,
// which the mixed form's inner solves see: 14 instead of 10 iterations at
// 512 x 512.)
// A plan that holds a range of the windows and has a reduce callback sums its
// share over the ranks (matvec does that for op 0).
void plan_degrees(Plan &P, cudaStream_t s) {
    k_fill<<<kRedBlocks, kRedThreads, 0, s>>>(P.t, P.N, 1.0);
    NLH_CHECK_LAUNCH();
    if (P.precision & 1) matvec(P, 0, NLH_FP64, 0.0, P.t, P.d64, nullptr, nullptr, s);
    if (P.precision & 2) matvec(P, 0, NLH_FP32, 0.0, P.t, P.d32, nullptr, nullptr, s);
    if (P.precision & 4) matvec(P, 0, NLH_DF32, 0.0, P.t, P.ddf, nullptr, nullptr, s);
}

static void build_plan(Plan &P, const nlh_plan_desc &desc, const double *features,
                       cudaStream_t s) {
    NLH_CUDA(cudaGetDevice(&P.device));
    P.N = desc.N;
    P.D = desc.D;
    P.M = desc.M;
    P.n = desc.n_os;
    P.m = desc.m;
    P.W2 = 2 * desc.m;
    P.precision = desc.precision;
    P.sigma = desc.sigma;
    P.kmax = desc.max_items_pts > 0 ? desc.max_items_pts : 64;
    P.unit_points = desc.unit_points > 0 ? desc.unit_points : kUnitPoints;
    for (int a = 0; a < 3; ++a) {
        NLH_REQUIRE(desc.team[a] >= 0 && desc.team[a] <= 2, "nlh_plan_create: team[%d]=%d", a,
                    desc.team[a]);
        P.team[a] = desc.team[a];
    }
    // the plan's windows: all of them, or the range [window_first,
    // window_first + window_count) of the list (the torus map is taken over
    // the whole list, so that plans of complementary ranges sum to the
    // operator of all windows)
    const int L_all = desc.L;
    const int wf = desc.window_count > 0 ? desc.window_first : 0;
    const int L = desc.window_count > 0 ? desc.window_count : L_all;
    P.L = L;
    P.L_norm = L_all;
    P.window_first = wf;
    P.reduce_fn = desc.reduce;
    P.reduce_ctx = desc.reduce_ctx;
    P.windows.assign(desc.windows, desc.windows + 3 * L_all);
    const int64_t N = P.N;

    int *d_win = P.alloc<int>(3 * L_all);
    NLH_CUDA(cudaMemcpyAsync(d_win, P.windows.data(), sizeof(int) * 3 * L_all,
                             cudaMemcpyHostToDevice, s));

    // per-window, per-dim ranges -> torus map
    const int nb = 152;
    double *part = P.alloc<double>((size_t)3 * L_all * nb * 2);
    double *mm = P.alloc<double>((size_t)3 * L_all * 2);
    k_minmax_partial<<<dim3(nb, 3 * L_all), 256, 0, s>>>(features, N, P.D, d_win, part);
    NLH_CHECK_LAUNCH();
    k_minmax_final<<<3 * L_all, 32, 0, s>>>(part, nb, mm);
    NLH_CHECK_LAUNCH();
    std::vector<double> hmm(6 * L_all), center(3 * L_all);
    NLH_CUDA(cudaMemcpyAsync(hmm.data(), mm, sizeof(double) * 6 * L_all, cudaMemcpyDeviceToHost,
                             s));
    NLH_CUDA(cudaStreamSynchronize(s));
    double R = 0.0;
    for (int c = 0; c < 3 * L_all; ++c) {
        NLH_REQUIRE(std::isfinite(hmm[2 * c]) && std::isfinite(hmm[2 * c + 1]),
                    "features contain non-finite values");
        center[c] = 0.5 * (hmm[2 * c] + hmm[2 * c + 1]);
        R = std::max(R, hmm[2 * c + 1] - hmm[2 * c]);
    }
    if (!(R > 0.0)) R = 1.0;
    P.R = R;
    if (desc.nfft_eps > 0.0) {
        auto_params(P.sigma, R, desc.nfft_eps, desc.m, (int64_t)L * N, L, P.M, P.n, P.m,
                    P.fill);
        P.W2 = 2 * P.m;
    } else {
        P.fill = desc.torus_fill > 0.0 ? desc.torus_fill : choose_fill(P.sigma, R, P.M);
    }
    P.scale = P.fill / R;
    P.kb_beta = M_PI * P.m * (2.0 - (double)P.M / P.n);
    {
        const WinSets ws = fit_window(P.m, P.kb_beta);
        P.wp32 = ws.f32;
        P.wp64 = ws.f64;
        P.wpdf = ws.fdf;
        // staged tables for the kernels' shared-memory copies: FP64 {E_k, O_k}
        // per (j, k), then double-float {E hi, O hi, E lo, O lo} per (j, k)
        std::vector<float4> st(2 * kWinStageBytes / 16, make_float4(0.f, 0.f, 0.f, 0.f));
        double2 *st64 = reinterpret_cast<double2 *>(st.data());
        for (int j = 0; j < kWinHalfMax; ++j)
            for (int k = 0; k < kWinK64; ++k)
                st64[j * kWinK64 + k] = make_double2(ws.f64.c[j][0][k], ws.f64.c[j][1][k]);
        float4 *stdf = st.data() + kWinStageBytes / 16;
        for (int j = 0; j < kWinHalfMax; ++j)
            for (int k = 0; k < kWinK64; ++k)
                stdf[j * kWinK64 + k] = make_float4(ws.fdf.hi[j][0][k], ws.fdf.hi[j][1][k],
                                                    ws.fdf.lo[j][0][k], ws.fdf.lo[j][1][k]);
        P.wstage = P.alloc<float4>(st.size());
        NLH_CUDA(cudaMemcpyAsync(P.wstage, st.data(), sizeof(float4) * st.size(),
                                 cudaMemcpyHostToDevice, s));
        NLH_CUDA(cudaStreamSynchronize(s));  // the host table is a local
    }
    const int n = P.n;
    const int64_t n3 = (int64_t)n * n * n;
    double *d_center = P.alloc<double>(3 * L_all);
    NLH_CUDA(cudaMemcpyAsync(d_center, center.data(), sizeof(double) * 3 * L_all,
                             cudaMemcpyHostToDevice, s));

    // grid coordinates, cell keys and per-cell counts (the plan's windows)
    const int64_t LN = (int64_t)L * N;
    double *u = nullptr;
    int *keys = nullptr, *hist = nullptr, *start = nullptr, *cnt = nullptr, *ioff = nullptr,
        *sums = nullptr, *scal = nullptr;
    NLH_CUDA(cudaMallocAsync(&u, sizeof(double) * LN * 3, s));
    std::vector<void *> tmp{u};
    auto tmp_alloc = [&](int **ptr, size_t count) {
        NLH_CUDA(cudaMallocAsync((void **)ptr, sizeof(int) * std::max<size_t>(count, 1), s));
        tmp.push_back(*ptr);
    };
    try {
        const int64_t ncells = (int64_t)L * n3;
        tmp_alloc(&keys, LN);
        tmp_alloc(&hist, ncells);
        tmp_alloc(&start, ncells);
        tmp_alloc(&cnt, ncells);
        tmp_alloc(&ioff, ncells);
        tmp_alloc(&sums, div_up(ncells, kScanTile) + 1);
        tmp_alloc(&scal, 2);
        NLH_CUDA(cudaMemsetAsync(hist, 0, sizeof(int) * ncells, s));
        NLH_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 2, s));
        const int gb = 152 * 8;
        k_cell_keys<<<gb, 256, 0, s>>>(features, N, P.D, L, d_win + 3 * wf, d_center + 3 * wf,
                                       P.scale, n, u, keys, hist);
        NLH_CHECK_LAUNCH();
        exclusive_scan_dev(hist, start, ncells, s, sums, scal);
        P.perm = P.alloc<int32_t>(LN);
        NLH_CUDA(cudaMemcpyAsync(cnt, start, sizeof(int) * ncells, cudaMemcpyDeviceToDevice, s));
        k_scatter<<<gb, 256, 0, s>>>(keys, N, L, n3, cnt, P.perm);
        NLH_CHECK_LAUNCH();
        k_item_counts<<<gb, 256, 0, s>>>(hist, ncells, P.kmax, cnt, scal + 1);
        NLH_CHECK_LAUNCH();
        int occ = 0;  // read with the synchronisation of the scan below
        NLH_CUDA(cudaMemcpyAsync(&occ, scal + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        P.n_items = exclusive_scan(P, cnt, ioff, ncells, s, sums, scal);
        P.items = P.alloc<int4>(P.n_items);
        k_emit_items<<<gb, 256, 0, s>>>(hist, start, ioff, ncells, n, P.kmax, P.items);
        NLH_CHECK_LAUNCH();
        build_units(P, s);
        if (desc.image) {
            // coordinates from the image: its copy, the patch offsets and the
            // torus map of the plan's windows (u = A x + B, the map
            // (s (x - c) + 0.5) n of k_cell_keys expanded)
            const int Pw = 2 * desc.patch_radius + 1;
            P.coords_image = 1;
            P.img_n1 = desc.image_n1;
            P.img_n2 = desc.image_n2;
            P.img_pad = desc.patch_pad;
            if (P.precision & 5) {
                P.img64 = P.alloc<double>(N);
                NLH_CUDA(cudaMemcpyAsync(P.img64, desc.image, sizeof(double) * N,
                                         cudaMemcpyDeviceToDevice, s));
            }
            if (P.precision & 2) {
                P.img2 = P.alloc<float2>(N);
                k_split_image<<<gb, 256, 0, s>>>(desc.image, N, P.img2);
                NLH_CHECK_LAUNCH();
            }
            std::vector<int4> off(3 * L);
            std::vector<double> hB(3 * L);
            std::vector<float2> hBdf(3 * L);
            P.cA = P.scale * n;
            P.cAdf = make_float2((float)P.cA, (float)(P.cA - (double)(float)P.cA));
            for (int l = 0; l < L; ++l)
                for (int t = 0; t < 3; ++t) {
                    const int k = P.windows[3 * (wf + l) + t];
                    off[3 * l + t] = k < 0 ? make_int4(1, 0, 0, 0)
                                           : make_int4(0, k / Pw - desc.patch_radius,
                                                       k % Pw - desc.patch_radius, 0);
                    const double B = (0.5 - P.scale * center[3 * (wf + l) + t]) * n;
                    hB[3 * l + t] = B;
                    hBdf[3 * l + t] = make_float2((float)B, (float)(B - (double)(float)B));
                }
            P.coff = P.alloc<int4>(3 * L);
            P.cB = P.alloc<double>(3 * L);
            P.cBdf = P.alloc<float2>(3 * L);
            NLH_CUDA(cudaMemcpyAsync(P.coff, off.data(), sizeof(int4) * 3 * L,
                                     cudaMemcpyHostToDevice, s));
            NLH_CUDA(cudaMemcpyAsync(P.cB, hB.data(), sizeof(double) * 3 * L,
                                     cudaMemcpyHostToDevice, s));
            NLH_CUDA(cudaMemcpyAsync(P.cBdf, hBdf.data(), sizeof(float2) * 3 * L,
                                     cudaMemcpyHostToDevice, s));
            NLH_CUDA(cudaStreamSynchronize(s));  // the host tables are locals
        } else {
            // cell offsets in sorted order (the low parts for the FP64-accurate paths)
            P.yhi = P.alloc<float>((size_t)LN * 3);
            if (P.precision & 5) P.ylo = P.alloc<float>((size_t)LN * 3);
            k_offsets<<<gb, 256, 0, s>>>(P.perm, u, N, L, P.yhi, P.ylo);
            NLH_CHECK_LAUNCH();
        }
        P.occupied = occ;
    } catch (...) {
        for (void *ptr : tmp) cudaFreeAsync(ptr, s);
        throw;
    }
    for (void *ptr : tmp) cudaFreeAsync(ptr, s);

    // tables, grids, outputs, solver workspace
    if (P.precision & 5) {  // FP64 and double-float paths share FP64 grids and tables
        P.tab64 = P.alloc<double>(n);
        P.tw64 = P.alloc<double2>(n / 2);
        P.gridA64 = P.alloc<double>((size_t)L * n3);
        P.gridB64 = P.alloc<double>((size_t)L * n3);
        NLH_CUDA(cudaMemsetAsync(P.gridA64, 0, sizeof(double) * L * n3, s));
    }
    if (P.precision & 1) P.d64 = P.alloc<double>(N);
    if (P.precision & 4) {
        P.ddf = P.alloc<double>(N);
        P.tabdf = P.alloc<float2>(n);
        P.twdf = P.alloc<float4>(n / 2);
    }
    if (P.precision & 2) {
        P.tab32 = P.alloc<float>(n);
        P.tw32 = P.alloc<float2>(n / 2);
        P.gridA32 = P.alloc<float>((size_t)L * n3);
        P.gridB32 = P.alloc<float>((size_t)L * n3);
        NLH_CUDA(cudaMemsetAsync(P.gridA32, 0, sizeof(float) * L * n3, s));
        P.d32 = P.alloc<double>(N);
    }
    P.yacc = P.alloc<double>(N);
    NLH_CUDA(cudaMemsetAsync(P.yacc, 0, sizeof(double) * N, s));
    P.w = P.alloc<double>(N);
    P.r = P.alloc<double>(N);
    P.p = P.alloc<double>(N);
    P.q = P.alloc<double>(N);
    P.t = P.alloc<double>(N);
    P.rhs = P.alloc<double>(N);
    P.pinv = P.alloc<double>(N);
    P.x0 = P.alloc<double>(N);
    P.cbuf = P.alloc<double>(N);
    P.partials = P.alloc<double>((size_t)kRedBlocks * 12 + kPqSlots);
    P.st = P.alloc<SolveState>(1);
    P.err = P.alloc<int>(1);
    NLH_CUDA(cudaMemsetAsync(P.err, 0, sizeof(int), s));
    P.unit_ctr = P.alloc<int>(2);
    NLH_CUDA(cudaMemsetAsync(P.unit_ctr, 0, sizeof(int) * 2, s));
    P.hist = P.alloc<double>(kMaxHist);
    take_pinned(P);
    plan_tables(P, s);
    plan_degrees(P, s);
    check_device_error(P, s);
    fetch_unit_count(P, s);
}

}  // namespace nlh

using namespace nlh;

extern "C" {

const char *nlh_last_error(void) { return g_err.c_str(); }

const char *nlh_version(void) { return "nlh 0.1 (sm_103a)"; }

nlh_status nlh_patch_features(const double *image, int n1, int n2, int radius, int pad,
                              double *features, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(image && features, "nlh_patch_features: NULL pointer");
        NLH_REQUIRE(n1 >= 1 && n2 >= 1 && radius >= 0 && radius <= 16,
                    "nlh_patch_features: bad sizes n1=%d n2=%d radius=%d", n1, n2, radius);
        NLH_REQUIRE(pad == 0 || pad == 1, "nlh_patch_features: pad must be 0 or 1");
        cudaStream_t s = (cudaStream_t)stream;
        int64_t total = (int64_t)n1 * n2 * (2 * radius + 1) * (2 * radius + 1);
        int blocks = (int)std::min<int64_t>(div_up(total, 256), 152 * 16);
        k_patch_features<<<blocks, 256, 0, s>>>(image, n1, n2, radius, pad, features);
        NLH_CHECK_LAUNCH();
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_create(nlh_plan *out, const nlh_plan_desc *desc, const double *features,
                           void *stream) {
    clear_error();
    nlh_plan_s *P = nullptr;
    try {
        NLH_REQUIRE(out && desc && features && desc->windows, "nlh_plan_create: NULL pointer");
        *out = nullptr;
        const nlh_plan_desc &d = *desc;
        NLH_REQUIRE(d.N >= 2 && d.N <= (int64_t)1 << 30, "nlh_plan_create: N=%lld out of range",
                    (long long)d.N);
        NLH_REQUIRE(d.D >= 1 && d.L >= 1 && d.L <= 64, "nlh_plan_create: D=%d L=%d", d.D, d.L);
        NLH_REQUIRE(d.nfft_eps >= 0.0 && d.nfft_eps < 0.1, "nlh_plan_create: nfft_eps=%g",
                    d.nfft_eps);
        if (d.nfft_eps == 0.0) {
            NLH_REQUIRE(d.n_os >= 32 && d.n_os <= 256 && (d.n_os & (d.n_os - 1)) == 0,
                        "nlh_plan_create: n_os=%d must be a power of two in [32, 256]", d.n_os);
            NLH_REQUIRE(d.M >= 4 && d.M <= d.n_os && d.M % 2 == 0,
                        "nlh_plan_create: M=%d must be even, 4 <= M <= n_os", d.M);
            NLH_REQUIRE(d.m >= 2 && d.m <= 8 && 2 * d.m < d.n_os, "nlh_plan_create: m=%d", d.m);
        } else {
            NLH_REQUIRE(d.m == 0 || (d.m >= 2 && d.m <= 8), "nlh_plan_create: m=%d", d.m);
        }
        NLH_REQUIRE(d.sigma > 0.0 && std::isfinite(d.sigma), "nlh_plan_create: sigma=%g",
                    d.sigma);
        NLH_REQUIRE(d.precision >= 1 && d.precision <= 7, "nlh_plan_create: precision=%d",
                    d.precision);
        NLH_REQUIRE(d.torus_fill >= 0.0 && d.torus_fill < 1.0, "nlh_plan_create: torus_fill=%g",
                    d.torus_fill);
        if (d.image)
            NLH_REQUIRE(d.image_n1 >= 1 && d.image_n2 >= 1 &&
                            (int64_t)d.image_n1 * d.image_n2 == d.N && d.patch_radius >= 0 &&
                            (d.patch_pad == 0 || d.patch_pad == 1) &&
                            (int64_t)(2 * d.patch_radius + 1) * (2 * d.patch_radius + 1) == d.D,
                        "nlh_plan_create: image %dx%d, radius %d, pad %d do not match N=%lld, "
                        "D=%d",
                        d.image_n1, d.image_n2, d.patch_radius, d.patch_pad, (long long)d.N,
                        d.D);
        NLH_REQUIRE(d.window_count >= 0 && d.window_first >= 0 &&
                        (d.window_count == 0 || d.window_first + d.window_count <= d.L),
                    "nlh_plan_create: window range [%d, %d + %d) outside the %d windows",
                    d.window_first, d.window_first, d.window_count, d.L);
        NLH_REQUIRE((int64_t)(d.window_count > 0 ? d.window_count : d.L) * d.N <
                        ((int64_t)1 << 31),
                    "nlh_plan_create: L*N too large");
        for (int i = 0; i < 3 * d.L; ++i)
            NLH_REQUIRE(d.windows[i] >= -1 && d.windows[i] < d.D,
                        "nlh_plan_create: windows[%d]=%d out of range", i, d.windows[i]);
        retain_pool_memory();
        prepare_nfft_kernels();
        P = new nlh_plan_s();
        static std::atomic<uint64_t> serials{0};
        P->serial = ++serials;
        P->stream = (cudaStream_t)stream;
        build_plan(*P, d, features, (cudaStream_t)stream);
        *out = P;
        return NLH_OK;
    } catch (Failure &f) {
        delete P;
        return f.st;
    } catch (std::bad_alloc &) {
        delete P;
        set_error("nlh_plan_create: host allocation failed");
        return NLH_ERR_OOM;
    }
}

nlh_status nlh_plan_set_sigma(nlh_plan plan, double sigma, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(plan, "nlh_plan_set_sigma: NULL plan");
        NLH_REQUIRE(sigma > 0.0 && std::isfinite(sigma), "nlh_plan_set_sigma: sigma=%g", sigma);
        cudaStream_t s = (cudaStream_t)stream;
        plan->stream = s;
        plan->sigma = sigma;
        plan_tables(*plan, s);
        plan_degrees(*plan, s);
        check_device_error(*plan, s);
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_get_degrees(nlh_plan plan, double *d, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(plan && d, "nlh_plan_get_degrees: NULL pointer");
        const double *src = (plan->precision & 1) ? plan->d64
                            : (plan->precision & 4) ? plan->ddf : plan->d32;
        NLH_CUDA(cudaMemcpyAsync(d, src, sizeof(double) * plan->N, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_get_info(nlh_plan plan, nlh_plan_info *info) {
    clear_error();
    try {
        NLH_REQUIRE(plan && info, "nlh_plan_get_info: NULL pointer");
        info->N = plan->N;
        info->L = plan->L;
        info->M = plan->M;
        info->n_os = plan->n;
        info->m = plan->m;
        info->precision = plan->precision;
        info->sigma = plan->sigma;
        info->torus_fill = plan->fill;
        info->scale = plan->scale;
        info->sigma_torus = plan->sigma * plan->scale;
        info->max_range = plan->R;
        info->n_items = plan->n_items;
        info->n_units = plan->n_units;
        info->max_items_pts = plan->kmax;
        info->unit_points = plan->unit_points;
        for (int a = 0; a < 3; ++a) info->team[a] = plan->team[a];
        info->window_first = plan->window_first;
        info->coords_from_image = plan->coords_image;
        info->window_count = plan->L;
        info->occupied_cells = plan->occupied;
        error_estimates(plan->sigma, plan->R, plan->fill, plan->M, &info->est_trunc_err,
                        &info->est_alias_err);
        info->device_bytes = plan->bytes;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_retile(nlh_plan plan, int max_items_pts, int unit_points, void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(plan, "nlh_plan_retile: NULL plan");
        NLH_REQUIRE(max_items_pts >= 1 && max_items_pts <= 4096,
                    "nlh_plan_retile: max_items_pts=%d", max_items_pts);
        NLH_REQUIRE(unit_points >= 1 && unit_points <= (1 << 20), "nlh_plan_retile: unit_points=%d",
                    unit_points);
        cudaStream_t s = (cudaStream_t)stream;
        plan->stream = s;
        retile(*plan, max_items_pts, unit_points, s);
        // degrees in the new summation order (L 1 = 0 to rounding again)
        plan_degrees(*plan, s);
        plan->pb2_sigma = -1.0;
        NLH_CUDA(cudaStreamSynchronize(s));
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_set_team(nlh_plan plan, int arith, int shape) {
    clear_error();
    try {
        NLH_REQUIRE(plan, "nlh_plan_set_team: NULL plan");
        NLH_REQUIRE(arith >= 0 && arith <= 2 && shape >= 0 && shape <= 2,
                    "nlh_plan_set_team: arith=%d shape=%d", arith, shape);
        if (plan->team[arith] != shape) {
            // new summation order: drop the captured solve graphs and
            // recompute the degrees (on the plan's last stream)
            drop_graphs(*plan);
            plan->team[arith] = shape;
            plan_degrees(*plan, plan->stream);
            plan->pb2_sigma = -1.0;
            NLH_CUDA(cudaStreamSynchronize(plan->stream));
        }
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_autotune(nlh_plan plan, int precisions, int reps, int *best_kmax,
                             int *best_unit_points, int *best_team, double *best_ms,
                             void *stream) {
    clear_error();
    try {
        NLH_REQUIRE(plan, "nlh_plan_autotune: NULL plan");
        const int mask = precisions ? precisions : plan->precision;
        NLH_REQUIRE((mask & plan->precision) == mask && mask > 0,
                    "nlh_plan_autotune: precisions=%d not built", precisions);
        cudaStream_t s = (cudaStream_t)stream;
        plan->stream = s;
        Plan &P = *plan;
        const int r = reps > 0 ? reps : 3;
        // probe vector: the degree input (ones) is already in P.t
        k_fill<<<kRedBlocks, kRedThreads, 0, s>>>(P.t, P.N, 1.0);
        NLH_CHECK_LAUNCH();
        cudaEvent_t e0, e1;
        NLH_CUDA(cudaEventCreate(&e0));
        NLH_CUDA(cudaEventCreate(&e1));
        const int kmaxes[] = {32, 64, 128, 256};
        const int unitpts[] = {256, 512, 1024, 2048};
        const int nshapes = (P.W2 == 8 || P.W2 == 12) ? 3 : 1;
        double best = INFINITY;
        int bk = P.kmax, bu = P.unit_points;
        int bt[3] = {P.team[0], P.team[1], P.team[2]};
        for (int km : kmaxes)
            for (int up : unitpts) {
                retile(P, km, up, s);
                double ms_total = 0.0;
                int tt[3] = {P.team[0], P.team[1], P.team[2]};
                for (int prec = 0; prec < 3; ++prec) {
                    if (!(mask & (prec == NLH_FP64 ? 1 : prec == NLH_FP32 ? 2 : 4))) continue;
                    double best_shape = INFINITY;
                    for (int sh = 0; sh < nshapes; ++sh) {
                        P.team[prec] = sh;
                        matvec(P, 0, prec, 0.0, P.t, P.q, nullptr, nullptr, s);  // warm
                        NLH_CUDA(cudaEventRecord(e0, s));
                        for (int k = 0; k < r; ++k)
                            matvec(P, 0, prec, 0.0, P.t, P.q, nullptr, nullptr, s);
                        NLH_CUDA(cudaEventRecord(e1, s));
                        NLH_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        NLH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        if (ms / r < best_shape) {
                            best_shape = ms / r;
                            tt[prec] = sh;
                        }
                    }
                    ms_total += best_shape;
                }
                if (ms_total < best) {
                    best = ms_total;
                    bk = km;
                    bu = up;
                    for (int a = 0; a < 3; ++a) bt[a] = tt[a];
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        retile(P, bk, bu, s);
        for (int a = 0; a < 3; ++a) P.team[a] = bt[a];
        plan_degrees(P, s);
        P.pb2_sigma = -1.0;
        check_device_error(P, s);
        if (best_kmax) *best_kmax = bk;
        if (best_unit_points) *best_unit_points = bu;
        if (best_team)
            for (int a = 0; a < 3; ++a) best_team[a] = bt[a];
        if (best_ms) *best_ms = best;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_plan_destroy(nlh_plan plan) {
    clear_error();
    delete plan;
    return NLH_OK;
}

}  // extern "C"
