// common.cuh -- internals shared by the translation units of libnlh.
//
// Device data layout of a plan (all device arrays are owned by the plan):
//   perm     [L*N]   int32   sorted position s (window l = s / N) -> pixel
//   yhi, ylo [L*N][3] float  offset y = 2 f - 1 of each sorted point inside
//                             its grid cell, per dim, as a float and the
//                             float remainder (ylo only with an FP64-accurate
//                             path); the window weights are evaluated from
//                             these in the kernels (window.cuh)
//   items    [n_items] int4  {window << 16 | lz << 6 | ly << 3 | lx, tile,
//                             first sorted position, point count}: (lx, ly,
//                             lz) is the cell inside its kTile^3 tile; the
//                             points of one item share one grid cell, hence
//                             one stencil.  Items are ordered tile-major.
//   units    [n_units] int4  {window, tile (z*nt+y)*nt+x, first item, item
//                             count}: a run of items inside one tile with at
//                             most ~kUnitPoints points; one CTA per unit
//   gridA/B  [L][n][n][n]    oversampled grids, x fastest, per arithmetic
//                             (FP64 grids also serve double-float): A is
//                             spread into and cleared again by the first
//                             convolution pass, B holds the convolved grid
//   tab64/32 [n]             per-dim Fourier multiplier in bit-reversed order
//   tw64/32  [n/2]           FFT twiddles exp(-2 pi i j / n)
//   yacc     [N]             per-pixel sum over windows (zero between
//                             matvecs; the finishing pass clears it)
//   d64/d32/ddf [N]          degrees d = Gamma_full 1 of each NFFT arithmetic
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <map>
#include <vector>

#include "../../include/nlh.h"
#include "window.cuh"

namespace nlh {

void set_error(const char *fmt, ...);
void clear_error();

struct Failure {
    nlh_status st;
};

#define NLH_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            ::nlh::set_error("%s failed: %s (%s:%d)", #call,                   \
                             cudaGetErrorString(e_), __FILE__, __LINE__);      \
            throw ::nlh::Failure{e_ == cudaErrorMemoryAllocation ? NLH_ERR_OOM \
                                                                 : NLH_ERR_CUDA}; \
        }                                                                      \
    } while (0)

void count_launch();

#define NLH_CHECK_LAUNCH()                                                     \
    do {                                                                       \
        ::nlh::count_launch();                                                 \
        NLH_CUDA(cudaGetLastError());                                          \
    } while (0)

// Brackets the launches issued in its scope with CUDA events on stream s
// when profiling is enabled (profile.cu).
class ProfRange {
  public:
    ProfRange(int cls, cudaStream_t s);
    ~ProfRange();
    ProfRange(const ProfRange &) = delete;
    ProfRange &operator=(const ProfRange &) = delete;

  private:
    int idx_;
    cudaStream_t s_;
};

#define NLH_REQUIRE(cond, ...)                                                 \
    do {                                                                       \
        if (!(cond)) {                                                         \
            ::nlh::set_error(__VA_ARGS__);                                     \
            throw ::nlh::Failure{NLH_ERR_ARG};                                 \
        }                                                                      \
    } while (0)

// Device-side scalars of one Krylov solve.  Written only by block 0 of the
// kernel that owns each field (see solve.cu); read by every kernel.
struct SolveState {
    int done;        // 1 once converged, broken down or out of iterations
    int status;      // 0 running/converged, -4 breakdown
    int k;           // completed iterations
    int maxit;
    double tol;
    double bnorm;    // ||rhs||
    double bmean;    // mean(rhs) (deflated methods)
    double rz;       // r^T z of the current iterate
    double rz_old;   // copy made by the update kernel
    double rr;       // ||r||^2 of the current iterate
    double alpha;    // shift of A = alpha I + L
    // stagnation exit (stag > 0): the solve ends when the best residual so
    // far has not fallen by 30 % for `stag` iterations with the residual
    // within 8x of tol, or for 3 stag iterations anywhere (the operator's
    // rounding floor)
    int stag;
    int k_best;      // iteration of the last such fall
    double best;     // best relative residual so far (0: none yet)
};

constexpr int kMaxHist = 4096;
constexpr int kTile = 8;          // tile edge in grid cells (spread/interp units)
constexpr int kUnitPoints = 512;  // default points per work unit before a tile is split
constexpr int kUnitItems = 256;   // items per work unit (staged in shared memory)
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 608;   // 4 x 152 SMs; grid-stride loops beyond
constexpr int kPqSlots = 2 * kRedBlocks;  // block partials of x^T y from the interpolation

struct Plan {
    int64_t N = 0;
    int D = 0, L = 0, M = 0, n = 0, m = 0, W2 = 0, precision = 0, kmax = 64;
    int L_norm = 0;            // windows the kernel sum is normalised by (all windows)
    int window_first = 0;      // first window of the plan in the full list
    nlh_reduce_fn reduce_fn = nullptr;  // sums a range plan's share over ranks
    void *reduce_ctx = nullptr;
    int unit_points = kUnitPoints;
    int team[3] = {0, 0, 0};   // spreading team shape per arithmetic
    double *pb2 = nullptr;     // (d' - 1) / L for P_b' (d' = Gamma_full 1 at sigma / sqrt 2)
    double pb2_sigma = -1.0;   // sigma pb2 was computed for
    int pc_kind = 0;           // preconditioner of the current solve: 0 P_a, 1 P_b'
    double sigma = 0, fill = 0, scale = 0, R = 0, kb_beta = 0;
    int64_t n_items = 0, occupied = 0;
    std::vector<int32_t> windows;
    // device arrays
    int32_t *perm = nullptr;
    int4 *items = nullptr;
    int4 *units = nullptr;
    int64_t n_units = 0;          // host copy of the unit count (-1: on the device only)
    int64_t units_cap = 0;        // capacity of `units` (an upper bound of the count)
    float *yhi = nullptr, *ylo = nullptr;  // cell offsets of the sorted points
    WinPoly<float> wp32;          // window polynomials per arithmetic (kernel parameters)
    WinPoly<double> wp64;
    WinPoly<df32> wpdf;
    float4 *wstage = nullptr;     // device: staged FP64 then double-float coefficient tables
    double *tab64 = nullptr;
    float *tab32 = nullptr;
    double2 *tw64 = nullptr;
    float2 *tw32 = nullptr;
    float2 *tabdf = nullptr;      // double-float multiplier (hi, lo)
    float4 *twdf = nullptr;       // double-float twiddles (re hi, re lo, im hi, im lo)
    double *gridA64 = nullptr, *gridB64 = nullptr;
    float *gridA32 = nullptr, *gridB32 = nullptr;
    double *yacc = nullptr;       // [N] per-pixel sum over windows
    double *d64 = nullptr, *d32 = nullptr, *ddf = nullptr;
    // solver workspace
    double *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr,
           *t = nullptr, *rhs = nullptr, *pinv = nullptr, *x0 = nullptr, *cbuf = nullptr;
    double *partials = nullptr;   // kRedBlocks * 12 + kPqSlots doubles
    SolveState *st = nullptr;     // device
    int *err = nullptr;           // device error word (bounded waits that gave up)
    int *unit_ctr = nullptr;      // device [2]: next unit of spread / interpolation
    int *d_units = nullptr;       // device [1]: the unit count
    SolveState *st_host = nullptr; // pinned mirror
    double *red_host = nullptr;   // pinned, 3 * kRedBlocks residual partials
    std::map<int, cudaGraphExec_t> graphs;  // solve graphs (see solve.cu)
    // coordinates from the image (nlh_plan_desc.image) instead of stored
    // offsets: a copy of the image (FP64 for the FP64 and double-float
    // paths, a (hi, lo) float pair per pixel for FP32), per (window, dim)
    // the patch offset {zero dim, dr, dc, 0} and the torus map as
    // u = A x + B[l][t] (grid coordinate of a feature value x)
    int coords_image = 0;
    double *img64 = nullptr;
    float2 *img2 = nullptr;
    int img_n1 = 0, img_n2 = 0, img_pad = 0;
    int4 *coff = nullptr;
    double cA = 0.0;
    float2 cAdf = {0.f, 0.f};
    double *cB = nullptr;
    float2 *cBdf = nullptr;
    uint64_t serial = 0;          // unique per plan creation (batch graph keys)
    unsigned graph_epoch = 0;     // incremented whenever the solve graphs are dropped
    cudaStream_t capture_stream = nullptr;
    int device = 0;               // the device the plan was built on
    double *hist = nullptr;       // device, kMaxHist
    std::vector<void *> allocs;
    int64_t bytes = 0;
    // Device memory comes from the stream-ordered pool allocator on the
    // stream of the current call; it is released on the last such stream.
    cudaStream_t stream = nullptr;

    // Frees one array of `allocs` early (stream-ordered).
    void release(void *ptr) {
        for (size_t k = 0; k < allocs.size(); ++k)
            if (allocs[k] == ptr) {
                cudaFreeAsync(ptr, stream);
                allocs.erase(allocs.begin() + k);
                return;
            }
    }

    template <typename T> T *alloc(size_t count) {
        void *ptr = nullptr;
        if (count == 0) count = 1;
        NLH_CUDA(cudaMallocAsync(&ptr, count * sizeof(T), stream));
        allocs.push_back(ptr);
        bytes += (int64_t)(count * sizeof(T));
        return static_cast<T *>(ptr);
    }
    ~Plan();
};

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; result valid in thread 0.  blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 32 */) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        s = (lane < nw) ? sh[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// Every thread of the block gets sum_{j < nparts} parts[j * stride + off].
// Deterministic: fixed order per thread, fixed tree.
__device__ __forceinline__ double reduce_partials(const double *parts, int nparts,
                                                  int stride, int off,
                                                  double *sh) {
    double v = 0.0;
    for (int j = threadIdx.x; j < nparts; j += blockDim.x) v += parts[j * stride + off];
    v = block_sum(v, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    double out = sh[32];
    __syncthreads();
    return out;
}

// ---------------------------------------------------------------- host API (internal)
void plan_tables(Plan &P, cudaStream_t s);
// Resolves every NFFT kernel on the current device (once per device).
void prepare_nfft_kernels();
// First failed index check of the NFFT kernels since the last call (check
// id, index, bound, block, thread in info5; 0 = none), cleared; synchronous.
int nfft_check_take(int *info5);
void ensure_pb2(Plan &P, cudaStream_t s);
// Keep freed pool memory in the process (set once).
void retain_pool_memory();
// Throws Failure{NLH_ERR_CUDA} if an NFFT kernel's index check failed,
// Failure{NLH_ERR_TIMEOUT} if a kernel recorded a bounded wait that gave up
// (synchronises s).
void check_device_error(Plan &P, cudaStream_t s);
cudaStream_t take_capture_stream(int device);
void give_capture_stream(int device, cudaStream_t s);
void plan_degrees(Plan &P, cudaStream_t s);
// Destroy the cached solve graphs (after a change of tiling or launch shape).
void drop_graphs(Plan &P);
// alpha_dev (optional): read alpha from device memory instead of `alpha`.
void matvec(Plan &P, int op, int prec, double alpha, const double *x, double *y,
            double *partials, const int *done, cudaStream_t s,
            const double *alpha_dev = nullptr);

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Reflect padding of the patch features (Sec. 5): index -1 maps to 1 and
// n to n - 2 (repeatedly, for radii beyond the image).
__device__ __forceinline__ int reflect_index(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}


}  // namespace nlh

// The opaque handle of the C ABI is the plan itself.
struct nlh_plan_s : public nlh::Plan {};
