// nfft.cu -- the per-matvec NFFT fast Gauss transform (Sec. 3 of arXiv
// 2407.06834): for every window l,
//   spread   G_l[g] = sum_i v_i prod_d phi(g_d/n - x~_{i,d})      (adjoint NFFT
//                                                                 gridding)
//   convolve G'_l = IFFT(w .* FFT(G_l)) per axis (w: Gaussian coefficients
//            over the squared window transform, |k| < M/2)
//   interp   y_{l,i} = sum_g G'_l[g] prod_d phi(x~_{i,d} - g_d/n)  (NFFT)
// and the epilogue y = (1/L) sum_l y_l (= Gamma_full v), L v = d o v - y or
// (alpha I + L) v (Sec. 2.3, Eq. discretized-state), with the block partial
// sums of v^T y for CG.
//
// A matvec is spread (which gathers v through the sort permutation itself),
// three axis passes of the convolution (the first also clears the spread
// grid for the next matvec), the interpolation, which adds every window's
// value into a per-pixel sum, and one finishing pass over the pixels with
// the epilogue (a plan of one window finishes inside the interpolation).
// No per-point data is stored beyond the sort permutation and the points'
// offsets inside their grid cells: the window weights are evaluated in
// registers from those offsets (window.cuh).
//
// Work decomposition: points are sorted by grid cell; a work item is up to
// kmax points of one cell, which share one 2m x 2m x 2m stencil; a work unit
// is a run of items inside one 8^3-cell tile (one CTA at a time, persistent
// CTAs take units from a global counter).
#include "common.cuh"

#include <type_traits>
#include "df32.cuh"
#include "window.cuh"

#include <algorithm>
#include <mutex>

namespace nlh {

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<df32> { using type = cdf; };

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

// Storage of one arithmetic: R = element of the staged weight records, G =
// global grid element.  A record holds, per dim t, 2m values (R = T) or, for
// df32, 2m high parts followed by 2m low parts.
template <typename T> struct Num { using R = T; using G = T; static constexpr int kParts = 1; };
template <> struct Num<df32> { using R = float; using G = double; static constexpr int kParts = 2; };

template <typename T, int W2>
__device__ __forceinline__ const typename Num<T>::R *rec_line(const typename Num<T>::R *wp, int t) {
    return wp + t * Num<T>::kParts * W2;
}
template <typename T, int W2>
__device__ __forceinline__ T rec_val(const typename Num<T>::R *wp, int t, int j) {
    return wp[t * W2 + j];
}
template <int W2> struct RecDF {
    static __device__ __forceinline__ df32 get(const float *wp, int t, int j) {
        return df32(wp[t * 2 * W2 + j], wp[t * 2 * W2 + W2 + j]);
    }
};
#define NLH_REC_DF(W)                                                                  \
    template <>                                                                        \
    __device__ __forceinline__ df32 rec_val<df32, W>(const float *wp, int t, int j) {  \
        return RecDF<W>::get(wp, t, j);                                                \
    }
NLH_REC_DF(4)
NLH_REC_DF(6)
NLH_REC_DF(8)
NLH_REC_DF(10)
NLH_REC_DF(12)
NLH_REC_DF(14)
NLH_REC_DF(16)
#undef NLH_REC_DF

template <typename T, int W2>
__device__ __forceinline__ void rec_put(typename Num<T>::R *wp, int t, int j, T v) {
    wp[t * W2 + j] = v;
}
template <int W2> struct RecPutDF {
    static __device__ __forceinline__ void put(float *wp, int t, int j, df32 v) {
        wp[t * 2 * W2 + j] = v.hi;
        wp[t * 2 * W2 + W2 + j] = v.lo;
    }
};
#define NLH_RECPUT_DF(W)                                                                     \
    template <>                                                                              \
    __device__ __forceinline__ void rec_put<df32, W>(float *wp, int t, int j, df32 v) {      \
        RecPutDF<W>::put(wp, t, j, v);                                                       \
    }
NLH_RECPUT_DF(4)
NLH_RECPUT_DF(6)
NLH_RECPUT_DF(8)
NLH_RECPUT_DF(10)
NLH_RECPUT_DF(12)
NLH_RECPUT_DF(14)
NLH_RECPUT_DF(16)
#undef NLH_RECPUT_DF

// A team is NW warps; a CTA holds TPB teams.  Teams synchronise among
// themselves only (a warp sync, or a named barrier for multi-warp teams).
template <int NW>
__device__ __forceinline__ void team_sync(int team) {
    if (NW == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(32 * NW) : "memory");
    }
}

// Weight record of one point staged in shared memory: 3 x 2m values padded
// to a multiple of 16 bytes (vector loads of the x line).
template <typename T, int W2>
constexpr int padded_record() {
    using R = typename Num<T>::R;
    return ((3 * Num<T>::kParts * W2 * (int)sizeof(R) + 15) / 16) * 16 / (int)sizeof(R);
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__device__ __forceinline__ void tile_origin(int tile, int n, int &tx0, int &ty0, int &tz0) {
    const int nt = n / kTile;
    tx0 = (tile % nt) * kTile;
    ty0 = ((tile / nt) % nt) * kTile;
    tz0 = (tile / (nt * nt)) * kTile;
}

// Item record (see common.cuh): x = window << 16 | lz << 6 | ly << 3 | lx
// (cell offsets inside the tile), y = tile, z = first sorted position,
// w = point count.
__device__ __forceinline__ void item_local(int packed, int &lx, int &ly, int &lz) {
    lx = packed & 7;
    ly = (packed >> 3) & 7;
    lz = (packed >> 6) & 7;
}

// The (item, chunk) work list of one team inside a unit.  Items are taken
// dynamically from a CTA-wide counter in shared memory, so teams that draw
// small items take more of them.
struct ChunkCursor {
    int ii, c0, start, cnt, local;
    __device__ __forceinline__ bool valid() const { return ii >= 0; }
};

template <int NW>
__device__ __forceinline__ int fetch_item(int *s_next, int *s_slot, int team, int tid) {
    int idx = 0;
    if (NW == 1) {
        if (tid == 0) idx = atomicAdd(s_next, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
    } else {
        if (tid == 0) *s_slot = atomicAdd(s_next, 1);
        team_sync<NW>(team);
        idx = *s_slot;
        team_sync<NW>(team);
    }
    return idx;
}

__device__ __forceinline__ ChunkCursor make_cursor(const int4 *s_items, int ii, int nit) {
    if (ii >= nit) return ChunkCursor{-1, 0, 0, 0, 0};
    int4 it = s_items[ii];
    return ChunkCursor{ii, 0, it.z, it.w, it.x};
}

template <int NW, int CH>
__device__ __forceinline__ ChunkCursor next_chunk(const ChunkCursor &c, const int4 *s_items,
                                                  int nit, int *s_next, int *s_slot, int team,
                                                  int tid) {
    ChunkCursor d = c;
    d.c0 += CH;
    if (d.c0 < d.cnt) return d;
    return make_cursor(s_items, fetch_item<NW>(s_next, s_slot, team, tid), nit);
}

// Arithmetic on one x line of the stencil.  On the FP32 path a line of 2m
// values is held as m 64-bit registers, each a pair of floats, and updated
// with the packed fma.rn.f32x2 instruction; on the FP64 path it is scalar.
template <typename T, int W2> struct Line {
    T v[W2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int a = 0; a < W2; ++a) v[a] = T(0);
    }
    __device__ __forceinline__ void load(const T *src) {  // 16-byte aligned
#pragma unroll
        for (int a = 0; a < W2; a += 2) {
            const double2 q = *reinterpret_cast<const double2 *>(src + a);
            v[a] = q.x;
            v[a + 1] = q.y;
        }
    }
    __device__ __forceinline__ void from(const T (&w)[W2]) {
#pragma unroll
        for (int a = 0; a < W2; ++a) v[a] = w[a];
    }
    __device__ __forceinline__ void axpy(T s, const Line &w) {  // v += s w
#pragma unroll
        for (int a = 0; a < W2; ++a) v[a] = fma(s, w.v[a], v[a]);
    }
    __device__ __forceinline__ T dot(const Line &h) const {
        T in = T(0);
#pragma unroll
        for (int a = 0; a < W2; ++a) in = fma(v[a], h.v[a], in);
        return in;
    }
    __device__ __forceinline__ T get(int a) const { return v[a]; }
    __device__ __forceinline__ void load_cells(const T *row) {  // 2m consecutive cells
#pragma unroll
        for (int a = 0; a < W2; ++a) v[a] = row[a];
    }
};

template <int W2> struct Line<float, W2> {
    static_assert(W2 % 2 == 0, "even stencil");
    unsigned long long v[W2 / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) v[a] = 0ull;
    }
    __device__ __forceinline__ void load(const float *src) {  // 8-byte aligned
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) v[a] = reinterpret_cast<const unsigned long long *>(src)[a];
    }
    __device__ __forceinline__ void from(const float (&w)[W2]) {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) v[a] = pk_make(w[2 * a], w[2 * a + 1]);
    }
    __device__ __forceinline__ void axpy(float s, const Line &w) {
        const unsigned long long ss = pk_dup(s);
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a)
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(v[a]) : "l"(ss), "l"(w.v[a]));
    }
    __device__ __forceinline__ float dot(const Line &h) const {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a)
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(v[a]), "l"(h.v[a]));
        float lo, hi;
        pk_split(acc, lo, hi);
        return lo + hi;
    }
    __device__ __forceinline__ float get(int a) const {
        float lo, hi;
        pk_split(v[a / 2], lo, hi);
        return (a & 1) ? hi : lo;
    }
    __device__ __forceinline__ void load_cells(const float *row) {  // 2m consecutive cells
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) v[a] = pk_make(row[2 * a], row[2 * a + 1]);
    }
    // 2m consecutive cells from a 16-byte aligned row (2m a multiple of 4)
    __device__ __forceinline__ void load_cells_v4(const float *row) {
        static_assert(W2 % 4 == 0, "whole 16-byte groups");
#pragma unroll
        for (int a = 0; a < W2 / 4; ++a) {
            const ulonglong2 q = reinterpret_cast<const ulonglong2 *>(row)[a];
            v[2 * a] = q.x;
            v[2 * a + 1] = q.y;
        }
    }
};

template <int W2> struct Line<df32, W2> {
    static_assert(W2 % 2 == 0, "even stencil");
    unsigned long long h[W2 / 2], l[W2 / 2];  // packed (cell a, cell a+1) high / low parts
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) h[a] = l[a] = 0ull;
    }
    // src: 2m high parts followed by 2m low parts (8-byte aligned)
    __device__ __forceinline__ void load(const float *src) { load2(src, src + W2); }
    // high and low parts from separate rows (8-byte aligned)
    __device__ __forceinline__ void load2(const float *hi, const float *lo) {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) {
            h[a] = reinterpret_cast<const unsigned long long *>(hi)[a];
            l[a] = reinterpret_cast<const unsigned long long *>(lo)[a];
        }
    }
    __device__ __forceinline__ void from(const df32 (&w)[W2]) {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) {
            h[a] = pk_make(w[2 * a].hi, w[2 * a + 1].hi);
            l[a] = pk_make(w[2 * a].lo, w[2 * a + 1].lo);
        }
    }
    __device__ __forceinline__ void axpy(df32 s, const Line &w) {  // this += s w
        const unsigned long long sh = pk_dup(s.hi), nsh = pk_dup(-s.hi), nsl = pk_dup(-s.lo);
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) pk_df_axpy(h[a], l[a], sh, nsh, nsl, w.h[a], w.l[a]);
    }
    __device__ __forceinline__ df32 dot(const Line &x) const {  // sum_a this[a] x[a]
        unsigned long long sh = 0ull, sl = 0ull;
        const unsigned long long zero = 0ull;
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a)
            pk_df_axpy(sh, sl, h[a], pk_sub(zero, h[a]), pk_sub(zero, l[a]), x.h[a], x.l[a]);
        float h0, h1, l0, l1;
        pk_split(sh, h0, h1);
        pk_split(sl, l0, l1);
        return df32(h0, l0) + df32(h1, l1);
    }
    __device__ __forceinline__ df32 get(int a) const {
        float h0, h1, l0, l1;
        pk_split(h[a / 2], h0, h1);
        pk_split(l[a / 2], l0, l1);
        return (a & 1) ? df32(h1, l1) : df32(h0, l0);
    }
    __device__ __forceinline__ void load_cells(const df32 *row) {  // 2m consecutive cells
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) {
            const df32 c0 = row[2 * a], c1 = row[2 * a + 1];
            h[a] = pk_make(c0.hi, c1.hi);
            l[a] = pk_make(c0.lo, c1.lo);
        }
    }
};

// (y, z) stencil pairs owned by one thread: pair p = q + NTP k, where q is
// the thread's index among the NTP threads that share its x segment.  When
// NTP is a multiple of 2m every pair of a thread has the same y offset.
template <int W2, int NTP, int PPT>
struct Pairs {
    int b0, bb[PPT], cc[PPT];
    bool ok[PPT];
    static constexpr bool kSameB = (NTP % W2) == 0;
    __device__ __forceinline__ void init(int q) {
        b0 = q % W2;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            int p = q + NTP * k;
            ok[k] = p < W2 * W2;
            bb[k] = kSameB ? b0 : (ok[k] ? p % W2 : 0);
            cc[k] = ok[k] ? p / W2 : 0;
        }
    }
};

// One x segment (WS = 2m / SPLIT consecutive cells) of a point's weight
// line, from its staged record.
template <typename T, int W2, int WS>
__device__ __forceinline__ void load_segment(Line<T, WS> &w, const typename Num<T>::R *line,
                                             int seg) {
    if constexpr (Num<T>::kParts == 2) {
        w.load2(line + seg * WS, line + W2 + seg * WS);
    } else {
        w.load(line + seg * WS);
    }
}

// The offset y = 2 f - 1 of a point inside its grid cell (per dim), stored
// as a float and the float remainder; each arithmetic reads what it needs.
template <typename T> struct Offs;
template <> struct Offs<float> {
    static __device__ __forceinline__ float get(const float *hi, const float *, int64_t k) {
        return __ldg(hi + k);
    }
};
template <> struct Offs<double> {
    static __device__ __forceinline__ double get(const float *hi, const float *lo, int64_t k) {
        return (double)__ldg(hi + k) + (double)__ldg(lo + k);
    }
};
template <> struct Offs<df32> {
    static __device__ __forceinline__ df32 get(const float *hi, const float *lo, int64_t k) {
        return df32(__ldg(hi + k), __ldg(lo + k));
    }
};

template <typename T> __device__ __forceinline__ T from_double(double v) { return T(v); }
template <> __device__ __forceinline__ float from_double<float>(double v) { return (float)v; }

// Plan data every NFFT kernel reads (device pointers of the plan).
struct NfftArgs {
    const int4 *units;
    const int *n_units;  // device copy of the unit count
    int *unit_ctr;       // [0] next spreading unit, [1] next interpolation unit
    const int4 *items;
    const int *perm;     // sorted position -> pixel (window-major)
    const float *yhi, *ylo;  // [sorted position][3] cell offsets y = 2 f - 1
    int n, m;
    int L;               // windows of the plan (units' window index < L)
    int64_t N;           // pixels (permutation entries < N; sorted positions < L N)
    const float4 *wstage;  // staged window coefficients of the arithmetic (FP64, df32)
    // coordinates from the image (img64 or img2 non-NULL) instead of yhi, ylo
    const double *img64;   // FP64 image (FP64 and double-float paths)
    const float2 *img2;    // (hi, lo) pairs of the image (FP32 path)
    int n1, n2, pad;       // image rows, columns; 1 reflect, 0 zero padding
    const int4 *coff;      // [window][dim] {zero dim, dr, dc, 0}
    const double *cB;      // [window][dim] B of u = A x + B
    const float2 *cBdf;
    double cA;
    float2 cAdf;
};

// ---- the cell offset y = 2 (u - c) - 1 of a point in dim t, recomputed from
// the image: the patch value x of pixel `pix` at the window's dim offset
// (reflect or zero padding, as the patch features), its grid coordinate
// u = A x + B[l][t] (the torus map of the plan), and its cell c along t (the
// item's cell; a difference of more than half the grid is the torus
// wrap).  FP64 arithmetic for the FP64 and double-float paths (the result
// matches the plan's stored FP64 offsets to ~1e-14), double-float for FP32.
// Row and column of a pixel (one 32-bit division per point).
struct PixRC {
    int r, c;
};
__device__ __forceinline__ PixRC pix_rc(const NfftArgs &a, int pix) {
    const unsigned r = (unsigned)pix / (unsigned)a.n2;
    return PixRC{(int)r, pix - (int)r * a.n2};
}

__device__ __forceinline__ int patch_pixel(const NfftArgs &a, PixRC p, int4 o, bool &zero) {
    int rr = p.r + o.y, cc = p.c + o.z;
    zero = o.x != 0;
    if (a.pad == 1) {
        rr = reflect_index(rr, a.n1);
        cc = reflect_index(cc, a.n2);
    } else if (rr < 0 || rr >= a.n1 || cc < 0 || cc >= a.n2) {
        zero = true;
    }
    return zero ? 0 : rr * a.n2 + cc;
}

__device__ __forceinline__ double torus_frac(double f, int n) {
    if (f > 0.5 * n) return f - n;
    if (f < -0.5 * n) return f + n;
    return f;
}

template <typename T> struct ImageOffs;
template <> struct ImageOffs<double> {
    static __device__ __forceinline__ double get(const NfftArgs &a, int l, int t, PixRC p,
                                                 int cell) {
        bool zero;
        const int q = patch_pixel(a, p, __ldg(a.coff + 3 * l + t), zero);
        const double x = zero ? 0.0 : __ldg(a.img64 + q);
        const double u = fma(a.cA, x, __ldg(a.cB + 3 * l + t));
        return fma(2.0, torus_frac(u - (double)cell, a.n), -1.0);
    }
};
template <> struct ImageOffs<df32> {
    static __device__ __forceinline__ df32 get(const NfftArgs &a, int l, int t, PixRC p,
                                               int cell) {
        return df32(ImageOffs<double>::get(a, l, t, p, cell));
    }
};
template <> struct ImageOffs<float> {
    static __device__ __forceinline__ float get(const NfftArgs &a, int l, int t, PixRC p,
                                                int cell) {
        bool zero;
        const int q = patch_pixel(a, p, __ldg(a.coff + 3 * l + t), zero);
        const float2 xv = zero ? make_float2(0.f, 0.f) : __ldg(a.img2 + q);
        const float2 bv = __ldg(a.cBdf + 3 * l + t);
        const df32 u = df32(a.cAdf.x, a.cAdf.y) * df32(xv.x, xv.y) + df32(bv.x, bv.y);
        // u hi - c is exact (c and u hi are close); the low part follows
        float f = __fadd_rn(__fsub_rn(u.hi, (float)cell), u.lo);
        if (f > 0.5f * a.n) f -= (float)a.n;
        else if (f < -0.5f * a.n) f += (float)a.n;
        return __fmaf_rn(2.f, f, -1.f);
    }
};

// The offset of point-window `sp` (pixel at p, window l, cell c along dim
// t): stored, or recomputed from the image.
template <typename T>
__device__ __forceinline__ T point_offset(const NfftArgs &a, int64_t sp, int t, int l, PixRC p,
                                          int cell) {
    if (a.coff) return ImageOffs<T>::get(a, l, t, p, cell);
    return Offs<T>::get(a.yhi, a.ylo, 3 * sp + t);
}

// Index checks on the plan data the NFFT kernels read from memory (unit and
// item records, permutation entries) and on the shared-memory rows they
// derive from them.  A failed check records, library-wide, the first
// failure (check id, index, bound, block, thread), which the next
// synchronising call of any plan reports (nfft_check_take), and the access
// is skipped: corrupt plan data becomes an error status, never an
// out-of-range access.
__device__ int g_nfft_check[5];

__device__ __forceinline__ bool idx_ok(bool cond, int id, long long idx, long long bound) {
    if (cond) return true;
    if (atomicCAS(&g_nfft_check[0], 0, id) == 0) {
        g_nfft_check[1] = (int)idx;
        g_nfft_check[2] = (int)bound;
        g_nfft_check[3] = blockIdx.x;
        g_nfft_check[4] = threadIdx.x;
    }
    return false;
}

// Prefetch of the byte range [b0, b1) of an array of total_bytes bytes
// (16-byte aligned base) into L2 with one bulk prefetch, the range widened
// to 16-byte boundaries and clipped to the array.
__device__ __forceinline__ void prefetch_l2(const void *base, int64_t b0, int64_t b1,
                                            int64_t total_bytes) {
    const int64_t lo = b0 & ~(int64_t)15;
    int64_t hi = (b1 + 15) & ~(int64_t)15;
    const int64_t cap = total_bytes & ~(int64_t)15;
    if (hi > cap) hi = cap;
    if (lo < 0 || hi <= lo) return;
    const char *p = static_cast<const char *>(base) + lo;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)(hi - lo))
                 : "memory");
}

// The point data of a unit's sorted range (permutation entries and cell
// offsets), prefetched into L2 once the unit's items are staged, so that the
// spreading teams' later chunks find it there (4% on FP32 spreading at
// 2m = 12; the interpolation, which reads each point once per lane right
// after staging its tile, measured no gain).  One thread, once per unit.
__device__ __noinline__ void prefetch_unit(const NfftArgs &a, const int4 *s_items, int nit,
                                              bool lo_parts) {
    const int64_t first = s_items[0].z, end = (int64_t)s_items[nit - 1].z + s_items[nit - 1].w;
    const int64_t total = (int64_t)a.L * a.N;
    if (first < 0 || end > total || end <= first) return;
    prefetch_l2(a.perm, 4 * first, 4 * end, 4 * total);
    if (a.coff) return;  // coordinates from the image: no stored offsets
    prefetch_l2(a.yhi, 12 * first, 12 * end, 12 * total);
    if (lo_parts) prefetch_l2(a.ylo, 12 * first, 12 * end, 12 * total);
}

// ------------------------------------------------------------------ spreading
// Shared memory of a spreading CTA: the tile region (kTile + 2m - 1)^3, the
// unit's items, control words, one broadcast slot per team, and per team the
// weight records of one chunk of NT points.
template <typename T, int W2, int NW, int TPB>
struct SpreadSmem {
    static constexpr int NT = 32 * NW, E = kTile + W2 - 1, E3 = E * E * E;
    static constexpr int PWP = padded_record<T, W2>();
    static constexpr size_t tile = align16(sizeof(T) * E3);
    static constexpr size_t items_off = tile;
    static constexpr size_t ctl_off = items_off + sizeof(int4) * kUnitItems;  // [0] items, [1] unit
    static constexpr size_t stage_off = ctl_off + 16;  // double-float coefficients
    static constexpr size_t slots_off = stage_off + kWinStageBytes;
    static constexpr size_t team_bytes = align16(sizeof(typename Num<T>::R) * NT * PWP);
    static constexpr size_t teams_off = slots_off + align16(sizeof(int) * TPB);
    // FP32 with coordinates from the image: the three offsets of each
    // thread's point (per team); none for the other arithmetics, whose
    // larger tiles and records must leave room for 2 CTAs per SM
    static constexpr size_t offs_bytes =
        std::is_same<T, float>::value ? align16(sizeof(T) * 3 * NT) : 0;
    static constexpr size_t offs_off = teams_off + TPB * team_bytes;
    static constexpr size_t bytes = offs_off + TPB * offs_bytes;
};

// Persistent CTAs take units from a global counter (units are stored in
// decreasing size).  Per unit, each team takes items; per chunk of NT points
// of an item every thread reads one point (its pixel through the sort
// permutation, the input value there, its cell offsets), evaluates the
// point's 3 x 2m window weights and stages them; then each thread adds the
// chunk's points into its PPT (y, z) stencil pairs, each an x segment of
// 2m / SPLIT accumulators in registers (all points of an item share the
// stencil).  An item's accumulators are then added into the shared tile,
// and the tile into the global grid once (non-zero entries only).
//
// SPLIT = 2 halves the x lines: a team of NT threads then covers the
// 2m x 2m x 2 (pair, segment) units, NT / 2 threads per segment, which for
// 2m = 12 and NT = 96 is exactly 3 units per thread (full lines leave a
// quarter of a 64-thread team idle in the third pass).
template <typename T, int W2, int NW, int TPB, int MINB = 1, int SPLIT = 1>
__global__ void __launch_bounds__(32 * NW * TPB, MINB)
k_spread(const NfftArgs a, const typename PolyArg<T>::type wp, const double *__restrict__ x,
         typename Num<T>::G *__restrict__ grid, const int *__restrict__ done) {
    using R = typename Num<T>::R;
    using G = typename Num<T>::G;
    using SM = SpreadSmem<T, W2, NW, TPB>;
    constexpr int NT = SM::NT, NTP = NT / SPLIT, WS = W2 / SPLIT;
    constexpr int PPT = (W2 * W2 + NTP - 1) / NTP, PWP = SM::PWP;
    static_assert(NT % SPLIT == 0 && WS % 2 == 0, "x segments of an even number of cells");
    constexpr int E = SM::E, E3 = SM::E3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + SM::items_off);
    int *s_ctl = reinterpret_cast<int *>(smem_raw + SM::ctl_off);
    float4 *s_coef = reinterpret_cast<float4 *>(smem_raw + SM::stage_off);
    if (done && *done) return;
    if constexpr (!std::is_same<T, float>::value) win_stage(a.wstage, s_coef);
    // the interpolation of the previous matvec has finished (stream order)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.unit_ctr[1] = 0;
    const int team = threadIdx.x / NT, tid = threadIdx.x % NT;
    const int seg = SPLIT == 1 ? 0 : tid / NTP;
    R *rec = reinterpret_cast<R *>(smem_raw + SM::teams_off + team * SM::team_bytes);
    T *s_offs = reinterpret_cast<T *>(smem_raw + SM::offs_off + team * SM::offs_bytes);
    int *s_slot = reinterpret_cast<int *>(smem_raw + SM::slots_off) + team;
    Pairs<W2, NTP, PPT> pr;
    pr.init(tid % NTP);
    const int msk = a.n - 1, m = a.m;
    const int64_t n_pts = (int64_t)a.L * a.N;
    while (true) {
        __syncthreads();  // previous unit fully flushed
        if (threadIdx.x == 0) s_ctl[1] = atomicAdd(&a.unit_ctr[0], 1);
        __syncthreads();
        const int uidx = s_ctl[1];
        if (uidx >= *a.n_units) break;
        const int4 un = a.units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        if (!idx_ok(nit >= 1 && nit <= kUnitItems && l >= 0 && l < a.L, 1, nit, l)) break;
        int tx0, ty0, tz0;
        tile_origin(un.y, a.n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < E3; e += blockDim.x) S[e] = T(0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = a.items[it0 + e];
        if (threadIdx.x == 0) s_ctl[0] = TPB;
        __syncthreads();
        if (threadIdx.x == 0) prefetch_unit(a, s_items, nit, !std::is_same<T, float>::value);
        Line<T, WS> acc[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[k].zero();
        ChunkCursor cur = make_cursor(s_items, team, nit);
        while (cur.valid()) {
            const int cn = min(NT, cur.cnt - cur.c0);
            if (tid < cn) {  // this thread's point: value, weights -> record
                const int64_t sp = (int64_t)cur.start + cur.c0 + tid;
                bool ok = idx_ok(sp >= 0 && sp < n_pts, 2, sp, 0);
                const int pix = ok ? __ldg(a.perm + sp) : 0;
                ok = ok && idx_ok(pix >= 0 && pix < a.N, 3, pix, sp);
                const T v = ok ? from_double<T>(__ldg(x + pix)) : T(0);
                R *mine = rec + tid * PWP;
                int lx0, ly0, lz0;  // the point's cell (for offsets from the image)
                item_local(cur.local, lx0, ly0, lz0);
                const PixRC prc = pix_rc(a, ok ? pix : 0);
                const int64_t spo = ok ? sp : 0;
                if constexpr (std::is_same<T, float>::value) {
                    // FP32: the three offsets first, their loads in flight
                    // together, into this thread's shared slot
                    const T o0 = point_offset<T>(a, spo, 0, l, prc, tx0 + lx0);
                    const T o1 = point_offset<T>(a, spo, 1, l, prc, ty0 + ly0);
                    const T o2 = point_offset<T>(a, spo, 2, l, prc, tz0 + lz0);
                    T *so = s_offs + 3 * tid;
                    so[0] = o0;
                    so[1] = o1;
                    so[2] = o2;
                }
                // one dim at a time (keeps the Horner chains of the three
                // dims out of each other's registers; for the FP64-accurate
                // arithmetics the offset is formed inside the loop, which
                // keeps the compiler from holding the staged coefficients
                // in registers across it)
#pragma unroll 1
                for (int t = 0; t < 3; ++t) {
                    T w[W2];
                    T off;
                    if constexpr (std::is_same<T, float>::value) {
                        off = s_offs[3 * tid + t];
                    } else {
                        const int cell = t == 0 ? tx0 + lx0 : (t == 1 ? ty0 + ly0 : tz0 + lz0);
                        off = point_offset<T>(a, spo, t, l, prc, cell);
                    }
                    win_weights<W2>(wp, s_coef, off, w);
                    const T sc = t == 1 ? v : T(1);
#pragma unroll
                    for (int j = 0; j < W2; ++j) rec_put<T, W2>(mine, t, j, sc * w[j]);
                }
            }
            team_sync<NW>(team);
            if (!idx_ok(cn >= 0 && cn <= NT, 6, cn, NT)) break;
            for (int j = 0; j < cn; ++j) {
                const R *wpp = rec + j * PWP;
                Line<T, WS> wx;
                load_segment<T, W2, WS>(wx, rec_line<T, W2>(wpp, 0), seg);
                if (Pairs<W2, NTP, PPT>::kSameB) {
                    const T vb = rec_val<T, W2>(wpp, 1, pr.b0);  // v wy[b]
#pragma unroll
                    for (int k = 0; k < PPT; ++k)
                        if (pr.ok[k]) acc[k].axpy(vb * rec_val<T, W2>(wpp, 2, pr.cc[k]), wx);
                } else {
#pragma unroll
                    for (int k = 0; k < PPT; ++k)
                        if (pr.ok[k])
                            acc[k].axpy(rec_val<T, W2>(wpp, 1, pr.bb[k]) *
                                            rec_val<T, W2>(wpp, 2, pr.cc[k]),
                                        wx);
                }
            }
            if (cur.c0 + NT >= cur.cnt) {  // last chunk of the item: add into the tile
                int lx0, ly0, lz0;
                item_local(cur.local, lx0, ly0, lz0);
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (pr.ok[k]) {
                        const int ro =
                            ((lz0 + pr.cc[k]) * E + (ly0 + pr.bb[k])) * E + lx0 + seg * WS;
                        T *row = S + ro;
#pragma unroll
                        for (int q = 0; q < WS; ++q)
                            if (idx_ok(ro + q >= 0 && ro + q < E3, 4, ro + q, E3)) atomicAdd(&row[q], acc[k].get(q));
                    }
                    acc[k].zero();
                }
            }
            const ChunkCursor nxt = next_chunk<NW, NT>(cur, s_items, nit, s_ctl, s_slot, team, tid);
            team_sync<NW>(team);  // every read of the records is done before they are rewritten
            cur = nxt;
        }
        __syncthreads();
        G *g = grid + (int64_t)l * a.n * a.n * a.n;
        for (int e = threadIdx.x; e < E3; e += blockDim.x) {
            T val = S[e];
            if (val != T(0)) {
                int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
                int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                    gz = (tz0 - m + 1 + ez) & msk;
                if (idx_ok(e < E3, 5, e, E3)) atomicAdd(&g[((int64_t)gz * a.n + gy) * a.n + gx], (G)val);
            }
        }
    }
}

template <typename T> constexpr int spread_class() {
    return sizeof(T) == 4 ? NLH_K_SPREAD32 : (Num<T>::kParts == 2 ? NLH_K_SPREADDF : NLH_K_SPREAD64);
}
template <typename T> constexpr int interp_class() {
    return sizeof(T) == 4 ? NLH_K_INTERP32 : (Num<T>::kParts == 2 ? NLH_K_INTERPDF : NLH_K_INTERP64);
}

// ------------------------------------------------- interpolation + epilogue
// Epilogue of a matvec (Sec. 2.3, Eq. discretized-state): out = s for op 0,
// d o x - s for op 1, alpha x + d o x - s for op 2, where s = inv_l sum_l y_l
// over the plan's windows (inv_l = 1/L, or 1/(all windows) for a plan that
// holds a range of them).
struct Epilogue {
    const double *x, *d;
    double *y;
    double *yacc;      // [N] running sum over windows, zero between matvecs
    double *partials;  // [nparts] block partial sums of x^T out, or NULL
    int nparts;
    int L;             // windows of the plan
    double inv_l;
    int op;
    double alpha;
    const double *alpha_dev;  // alpha from device memory, or NULL
};

// One point per lane: a warp takes 32 consecutive (sorted) points of the
// unit, each lane finds its point's cell among the unit's items (binary
// search on the first sorted positions), evaluates its weights in registers
// and sums
//   y = sum_z wz[z] (wx . t_z),  t_z[x] = sum_y wy[y] S[z][y][x]
// over its stencil in the staged tile region, with no cross-lane reduction
// (consecutive points mostly share a cell, so their tile rows are the same
// addresses).  The value is added into the pixel's sum over windows (FP64
// atomic, so the order of the L additions, and the last bits of the result,
// may differ between calls); k_finish applies the epilogue.
constexpr int kInterpThreads = 256;

// Shared-memory layout of the interpolation tile.  FP32 with 2m a multiple
// of 4 stages 4 copies of the tile region, copy c shifted left by c cells
// (S_c[z][y][x] = S[z][y][x + c]) with rows padded to a multiple of 4
// cells, so that the 2m cells of any row from any start x0 are 2m / 4
// aligned 16-byte loads from copy x0 mod 4 (one shared load per 4
// multiply-adds instead of one per multiply-add).  Other arithmetics keep
// one unpadded copy.
template <typename T, int W2>
struct InterpTile {
    static constexpr int E = kTile + W2 - 1;
    static constexpr bool kVec = std::is_same<T, float>::value && W2 % 4 == 0;
    static constexpr int NC = kVec ? 4 : 1;
    static constexpr int EP = kVec ? ((kTile + W2 + 3) / 4) * 4 : E;  // row pitch
    static constexpr int COPY = E * E * EP;                            // cells per copy
    static constexpr size_t bytes = align16(sizeof(T) * NC * COPY);
};
// Interpolation CTAs whose lanes take two points of one cell each (the FP32
// 2m = 12 instance): every tile row read from shared memory serves both
// points' FMAs, half the row loads per FMA of one point per lane, which at
// 2m = 12 throttle the kernel's shared-memory instruction issue.  The
// points of an item are paired in order; an item with an odd count ends in
// a single point.
template <typename T, int W2>
__host__ __device__ constexpr bool interp_pairs() {
    return std::is_same<T, float>::value && W2 == 12;
}
// Threads of an interpolation CTA: 256 (the FP32 2m = 12 instance's 4-copy
// tile allows one CTA per SM; its paired lanes need ~2x the registers).
template <typename T, int W2>
constexpr int interp_threads() {
    return kInterpThreads;
}
// Interpolation CTAs that keep each lane's y and z window weights in shared
// memory ([k][lane]) instead of registers: the double-float ones (this
// removed the 2m = 12 instance's register spills, 4% faster).
template <typename T, int W2>
__host__ __device__ constexpr bool interp_smem_weights() {
    return Num<T>::kParts == 2;
}

template <typename T, int W2, int NTH = kInterpThreads, int MINB = 1>
__global__ void __launch_bounds__(NTH, MINB)
k_interp(const NfftArgs a, const typename PolyArg<T>::type wp,
         const typename Num<T>::G *__restrict__ grid,
         const Epilogue ep, const int *__restrict__ done) {
    using G = typename Num<T>::G;
    using TL = InterpTile<T, W2>;
    constexpr int E = TL::E, E3 = E * E * E, EP = TL::EP, NC = TL::NC, COPY = TL::COPY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + TL::bytes);
    int *s_ctl = reinterpret_cast<int *>(s_items + kUnitItems);
    float4 *s_coef = reinterpret_cast<float4 *>(s_ctl + 4);
    // each lane's y and z weights in shared memory ([k][lane], conflict-free)
    // when interp_smem_weights, out of the registers of the stencil loop
    T *s_wy = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(s_coef) + kWinStageBytes);
    T *s_wz = s_wy + W2 * NTH;
    constexpr bool PAIR = interp_pairs<T, W2>();
    // first pair of each item and the unit's pair count (paired lanes)
    int *s_pst = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(s_wy) +
                                         (interp_smem_weights<T, W2>() ? 2 * W2 * sizeof(T) * NTH
                                                                       : 0));
    __shared__ double sh_red[33];
    if (done && *done) return;
    if constexpr (!std::is_same<T, float>::value) win_stage(a.wstage, s_coef);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int msk = a.n - 1, m = a.m;
    const double alpha = ep.alpha_dev ? *ep.alpha_dev : ep.alpha;
    double part = 0.0;
    while (true) {
        __syncthreads();  // previous unit done with the tile
        if (threadIdx.x == 0) s_ctl[0] = atomicAdd(&a.unit_ctr[1], 1);
        __syncthreads();
        const int uidx = s_ctl[0];
        if (uidx >= *a.n_units) break;
        const int4 un = a.units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        if (!idx_ok(nit >= 1 && nit <= kUnitItems && l >= 0 && l < a.L, 11, nit, l)) break;
        int tx0, ty0, tz0;
        tile_origin(un.y, a.n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = a.items[it0 + e];
        if constexpr (PAIR) {
            // warp 0: s_pst[e] = pairs of items before e, s_pst[nit] = all
            if (warp == 0) {
                int carry = 0;
                if (lane == 0) s_pst[0] = 0;
                for (int c = 0; c < nit; c += 32) {
                    const int e = c + lane;
                    const int v = e < nit ? (a.items[it0 + e].w + 1) >> 1 : 0;
                    int inc = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += u;
                    }
                    if (e < nit) s_pst[e + 1] = carry + inc;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
        }
        const G *g = grid + (int64_t)l * a.n * a.n * a.n;
        {
            constexpr int UNR = 8;
            for (int base = threadIdx.x; base < E3; base += blockDim.x * UNR) {
                G vals[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int e = base + u * blockDim.x;
                    vals[u] = G(0);
                    if (e < E3) {
                        const int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
                        const int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                                  gz = (tz0 - m + 1 + ez) & msk;
                        vals[u] = __ldg(&g[((int64_t)gz * a.n + gy) * a.n + gx]);
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int e = base + u * blockDim.x;
                    if (e < E3) {
                        if constexpr (NC == 1) {
                            S[e] = T(vals[u]);
                        } else {
                            const int ex = e % E, row = (e / E) * EP;
#pragma unroll
                            for (int c = 0; c < NC; ++c)
                                if (ex >= c) S[c * COPY + row + ex - c] = T(vals[u]);
                        }
                    }
                }
            }
        }
        __syncthreads();
        // epilogue: one window alone finishes the pixel here; with several
        // windows the value is added into the pixel's sum, which k_finish
        // turns into the output after every window is in
        auto finish = [&](int i, T acc) {
            const double val = (double)acc;
            if (ep.L > 1) {
                atomicAdd(&ep.yacc[i], val);
            } else {
                const double s = val * ep.inv_l;
                double out = s;
                const double xi = (ep.op != 0 || ep.partials) ? __ldg(ep.x + i) : 0.0;
                if (ep.op != 0) {
                    out = __ldg(ep.d + i) * xi - s;
                    if (ep.op == 2) out = fma(alpha, xi, out);
                }
                ep.y[i] = out;
                part = fma(xi, out, part);
            }
        };
        if constexpr (PAIR) {
            const int npairs = s_pst[nit];
            for (int q = warp * 32 + lane; q - lane < npairs; q += nwarp * 32) {
                if (q >= npairs) continue;
                int lo = 0, hi = nit - 1;  // the last item whose first pair is at or before q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_pst[mid] <= q) lo = mid; else hi = mid - 1;
                }
                const int4 itm = s_items[lo];
                const int o = 2 * (q - s_pst[lo]);
                const bool two = o + 1 < itm.w;
                const int sp1 = itm.z + o, sp2 = two ? sp1 + 1 : sp1;
                int lx0, ly0, lz0;
                item_local(itm.x, lx0, ly0, lz0);
                if (!idx_ok(sp1 >= 0 && sp2 < (int64_t)a.L * a.N && o < itm.w, 12, sp1, lo)) continue;
                const int i1 = __ldg(a.perm + sp1), i2 = __ldg(a.perm + sp2);
                if (!idx_ok(i1 >= 0 && i1 < a.N && i2 >= 0 && i2 < a.N, 14, i1, sp1)) continue;
                T wxa[W2], wy1[W2], wz1[W2], wy2[W2], wz2[W2];
                Line<T, W2> wx1, wx2, t1, t2, h;
                {
                    const PixRC prc = pix_rc(a, i1);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp1, 0, l, prc, tx0 + lx0), wxa);
                    wx1.from(wxa);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp1, 1, l, prc, ty0 + ly0), wy1);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp1, 2, l, prc, tz0 + lz0), wz1);
                }
                {
                    const PixRC prc = pix_rc(a, i2);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp2, 0, l, prc, tx0 + lx0), wxa);
                    wx2.from(wxa);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp2, 1, l, prc, ty0 + ly0), wy2);
                    win_weights<W2>(wp, s_coef, point_offset<T>(a, sp2, 2, l, prc, tz0 + lz0), wz2);
                }
                T acc1 = T(0), acc2 = T(0);
                const int cx = NC == 1 ? 0 : (lx0 & 3);
                const T *scopy = S + cx * COPY;
#pragma unroll 1
                for (int z = 0; z < W2; ++z) {
                    t1.zero();
                    t2.zero();
                    const int so = ((lz0 + z) * E + ly0) * EP + lx0 - cx;
                    if (!idx_ok(so >= 0 && so + (W2 - 1) * EP + W2 - 1 < COPY, 13, so, COPY)) break;
                    const T *srow = scopy + so;
#pragma unroll
                    for (int y = 0; y < W2; ++y) {
                        h.load_cells_v4(srow + y * EP);
                        t1.axpy(wy1[y], h);
                        t2.axpy(wy2[y], h);
                    }
                    // wz[z] by a select over the unrolled arrays (no local memory)
                    T w1 = wz1[0], w2 = wz2[0];
#pragma unroll
                    for (int k = 1; k < W2; ++k)
                        if (z == k) {
                            w1 = wz1[k];
                            w2 = wz2[k];
                        }
                    acc1 = fma(w1, wx1.dot(t1), acc1);
                    acc2 = fma(w2, wx2.dot(t2), acc2);
                }
                finish(i1, acc1);
                if (two) finish(i2, acc2);
            }
        } else {
            const int first = s_items[0].z;
            const int total = s_items[nit - 1].z + s_items[nit - 1].w - first;
            for (int p = warp * 32 + lane; p - lane < total; p += nwarp * 32) {
                if (p >= total) continue;
                const int sp = first + p;
                int lo = 0, hi = nit - 1;  // the last item starting at or before sp
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_items[mid].z <= sp) lo = mid; else hi = mid - 1;
                }
                int lx0, ly0, lz0;
                item_local(s_items[lo].x, lx0, ly0, lz0);
                if (!idx_ok(sp >= 0 && sp < (int64_t)a.L * a.N && lo >= 0 && lo < nit, 12, sp, lo)) continue;
                const int i = __ldg(a.perm + sp);
                if (!idx_ok(i >= 0 && i < a.N, 14, i, sp)) continue;
                T wxa[W2], wy[W2], wz[W2];
                const PixRC prc = pix_rc(a, i);
                const T o0 = point_offset<T>(a, sp, 0, l, prc, tx0 + lx0);
                const T o1 = point_offset<T>(a, sp, 1, l, prc, ty0 + ly0);
                const T o2 = point_offset<T>(a, sp, 2, l, prc, tz0 + lz0);
                win_weights<W2>(wp, s_coef, o0, wxa);
                win_weights<W2>(wp, s_coef, o1, wy);
                win_weights<W2>(wp, s_coef, o2, wz);
                Line<T, W2> wx, t, h;
                wx.from(wxa);
                T acc = T(0);
                constexpr bool SW = interp_smem_weights<T, W2>();
                if constexpr (SW) {
    #pragma unroll
                    for (int k = 0; k < W2; ++k) {
                        s_wy[k * NTH + threadIdx.x] = wy[k];
                        s_wz[k * NTH + threadIdx.x] = wz[k];
                    }
                }
                // the z loop stays rolled (the unrolled y loop is the work; a
                // fully unrolled stencil makes the compile very long)
                // the copy whose rows start 16-byte aligned at x = lx0 (one copy:
                // the plain tile)
                const int cx = NC == 1 ? 0 : (lx0 & 3);
                const T *scopy = S + cx * COPY;
    #pragma unroll 1
                for (int z = 0; z < W2; ++z) {
                    t.zero();
                    const int so = ((lz0 + z) * E + ly0) * EP + lx0 - cx;
                    if (!idx_ok(so >= 0 && so + (W2 - 1) * EP + W2 - 1 < COPY, 13, so, COPY)) break;
                    const T *srow = scopy + so;
    #pragma unroll
                    for (int y = 0; y < W2; ++y) {
                        if constexpr (NC == 1) {
                            h.load_cells(srow + y * EP);
                        } else {
                            h.load_cells_v4(srow + y * EP);
                        }
                        if constexpr (SW) t.axpy(s_wy[y * NTH + threadIdx.x], h);
                        else t.axpy(wy[y], h);
                    }
                    T wzz;
                    if constexpr (SW) {
                        wzz = s_wz[z * NTH + threadIdx.x];
                    } else {
                        // wz[z] by a select over the unrolled array (no local memory)
                        wzz = wz[0];
    #pragma unroll
                        for (int k = 1; k < W2; ++k)
                            if (z == k) wzz = wz[k];
                    }
                    acc = fma(wzz, wx.dot(t), acc);
                }
                finish(i, acc);
            }
        }
    }
    if (ep.partials && ep.L == 1) {
        const double bs = block_sum(part, sh_red);
        if (threadIdx.x == 0 && idx_ok(blockIdx.x < ep.nparts, 15, blockIdx.x, ep.nparts)) ep.partials[blockIdx.x] = bs;
        if (blockIdx.x == 0)
            for (int j = gridDim.x + threadIdx.x; j < ep.nparts; j += blockDim.x) ep.partials[j] = 0.0;
    }
}

// ------------------------------------------------------------------ grid convolution
// Circular convolution of one complex line of length n = 32 R held by a
// warp (element e at lane e % 32, register e / 32) with the real, even
// multiplier: a radix-2 decimation-in-frequency FFT (output in bit-reversed
// order), the multiply by the bit-reversed multiplier table, and the
// decimation-in-time inverse FFT (bit-reversed in, natural out).  Because
// the multiplier is real and even, the real and imaginary parts stay two
// independent convolved real lines.
template <typename T, int R>
__device__ __forceinline__ void conv_line(typename Vec2<T>::type (&xv)[R], const T *__restrict__ tab,
                                          const typename Vec2<T>::type *__restrict__ tw,
                                          int lane) {
    using C = typename Vec2<T>::type;
    constexpr int n = 32 * R;
    // forward DIF
#pragma unroll
    for (int h = n / 2; h >= 32; h >>= 1) {
        const int H = h / 32;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & H) == 0) {
                C p = xv[r], q = xv[r + H];
                xv[r] = cadd(p, q);
                int j = ((r % H) * 32 + lane) * (n / (2 * h));
                xv[r + H] = cmul(csub(p, q), tw[j]);
            }
        }
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const C w = tw[(lane & (h - 1)) * (n / (2 * h))];
        const bool upper = lane & h;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C o = cshfl(xv[r], h);
            xv[r] = upper ? cmul(csub(o, xv[r]), w) : cadd(xv[r], o);
        }
    }
    // multiply (table is in bit-reversed order, like the data)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        T f = tab[32 * r + lane];
        xv[r].x *= f;
        xv[r].y *= f;
    }
    // inverse DIT
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1) {
        const C w = tw[(lane & (h - 1)) * (n / (2 * h))];
        const bool upper = lane & h;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C mine = upper ? cmulc(xv[r], w) : xv[r];
            C o = cshfl(mine, h);
            xv[r] = upper ? csub(o, mine) : cadd(mine, o);
        }
    }
#pragma unroll
    for (int h = 32; h <= n / 2; h <<= 1) {
        const int H = h / 32;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & H) == 0) {
                int j = ((r % H) * 32 + lane) * (n / (2 * h));
                C q = cmulc(xv[r + H], tw[j]);
                C p = xv[r];
                xv[r] = cadd(p, q);
                xv[r + H] = csub(p, q);
            }
        }
    }
}

// One axis pass: one CTA = 16 grid lines along `axis`, staged through shared
// memory so that global loads and stores are contiguous rows; each warp
// convolves two real lines as one complex line.  The first axis pass reads
// the spread grid `src`, clears it for the next matvec and writes `dst`;
// the later passes work in place on `dst`.
template <typename T, int R>
__global__ void __launch_bounds__(256)
k_conv(typename Num<T>::G *__restrict__ src, typename Num<T>::G *__restrict__ dst, int axis,
       const T *__restrict__ tab, const typename Vec2<T>::type *__restrict__ tw,
       int *__restrict__ ctr_reset, const int *__restrict__ done) {
    using G = typename Num<T>::G;
    using C = typename Vec2<T>::type;
    constexpr int n = 32 * R, LPC = 16, PITCH = n + 1;
    __shared__ T S[LPC * PITCH];
    if (done && *done) return;
    // the spreading of this matvec has finished (stream order)
    if (ctr_reset && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ctr_reset = 0;
    const bool clear = src != dst;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    G *gs = src + (int64_t)blockIdx.y * n * n * n;
    G *gd = dst + (int64_t)blockIdx.y * n * n * n;
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
            const int64_t o = goff(j, e);
            S[j * PITCH + e] = T(gs[o]);
            if (clear) gs[o] = G(0);
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            const int64_t o = goff(j, e);
            S[j * PITCH + e] = T(gs[o]);
            if (clear) gs[o] = G(0);
        }
    }
    __syncthreads();

    C xv[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
        xv[r] = {S[(2 * warp) * PITCH + 32 * r + lane], S[(2 * warp + 1) * PITCH + 32 * r + lane]};
    conv_line<T, R>(xv, tab, tw, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        S[(2 * warp) * PITCH + 32 * r + lane] = xv[r].x;
        S[(2 * warp + 1) * PITCH + 32 * r + lane] = xv[r].y;
    }
    __syncthreads();
    if (axis == 0) {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q / n, e = q % n;
            gd[goff(j, e)] = (G)S[j * PITCH + e];
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            gd[goff(j, e)] = (G)S[j * PITCH + e];
        }
    }
}

// The x and y passes in one kernel: one CTA = one z plane of one window,
// staged whole in shared memory (n (n + 1) elements, rows padded against
// bank conflicts of the column pass), convolved along x (rows) and then
// along y (columns) by the CTA's warps two lines at a time, and written
// back once.  Reads the spread grid `src`, clears it for the next matvec
// and writes `dst`; the z pass (k_conv, axis 2) follows in place.
constexpr int kConvXYThreads = 512;
template <typename T>
constexpr size_t conv_xy_smem(int n) {
    return sizeof(T) * (size_t)n * (n + 1);
}

template <typename T, int R>
__global__ void __launch_bounds__(kConvXYThreads)
k_conv_xy(typename Num<T>::G *__restrict__ src, typename Num<T>::G *__restrict__ dst,
          const T *__restrict__ tab, const typename Vec2<T>::type *__restrict__ tw,
          int *__restrict__ ctr_reset, const int *__restrict__ done) {
    using G = typename Num<T>::G;
    using C = typename Vec2<T>::type;
    constexpr int n = 32 * R, PITCH = n + 1, NWARP = kConvXYThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    if (done && *done) return;
    // the spreading of this matvec has finished (stream order)
    if (ctr_reset && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ctr_reset = 0;
    const bool clear = src != dst;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t plane = ((int64_t)blockIdx.y * n + blockIdx.x) * n * n;  // (window, z)
    G *gs = src + plane;
    G *gd = dst + plane;
    for (int q = tid; q < n * n; q += kConvXYThreads) {
        const int y = q / n, x = q % n;
        S[y * PITCH + x] = T(gs[q]);
        if (clear) gs[q] = G(0);
    }
    __syncthreads();
    // x lines: rows 2 p and 2 p + 1 as one complex line
    for (int p = warp; p < n / 2; p += NWARP) {
        C xv[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            xv[r] = {S[(2 * p) * PITCH + 32 * r + lane], S[(2 * p + 1) * PITCH + 32 * r + lane]};
        conv_line<T, R>(xv, tab, tw, lane);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            S[(2 * p) * PITCH + 32 * r + lane] = xv[r].x;
            S[(2 * p + 1) * PITCH + 32 * r + lane] = xv[r].y;
        }
    }
    __syncthreads();
    // y lines: columns 2 p and 2 p + 1 as one complex line
    for (int p = warp; p < n / 2; p += NWARP) {
        C xv[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            xv[r] = {S[(32 * r + lane) * PITCH + 2 * p], S[(32 * r + lane) * PITCH + 2 * p + 1]};
        conv_line<T, R>(xv, tab, tw, lane);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            S[(32 * r + lane) * PITCH + 2 * p] = xv[r].x;
            S[(32 * r + lane) * PITCH + 2 * p + 1] = xv[r].y;
        }
    }
    __syncthreads();
    for (int q = tid; q < n * n; q += kConvXYThreads) {
        const int y = q / n, x = q % n;
        gd[q] = (G)S[y * PITCH + x];
    }
}

// ------------------------------------------------------------------ dispatch
template <typename T> constexpr int arith_index() {
    return std::is_same<T, df32>::value ? NLH_DF32 : (sizeof(T) == 8 ? NLH_FP64 : NLH_FP32);
}

template <typename T> typename PolyArg<T>::type win_poly(const Plan &) { return {}; }
template <> WinPoly<float> win_poly<float>(const Plan &P) { return P.wp32; }

template <typename T>
static NfftArgs nfft_args(const Plan &P) {
    NfftArgs a;
    a.units = P.units;
    a.n_units = P.d_units;
    a.unit_ctr = P.unit_ctr;
    a.items = P.items;
    a.perm = P.perm;
    a.yhi = P.yhi;
    a.ylo = P.ylo;
    a.img64 = P.img64;
    a.img2 = P.img2;
    a.n1 = P.img_n1;
    a.n2 = P.img_n2;
    a.pad = P.img_pad;
    a.coff = P.coords_image ? P.coff : nullptr;
    a.cB = P.cB;
    a.cBdf = P.cBdf;
    a.cA = P.cA;
    a.cAdf = P.cAdf;
    a.n = P.n;
    a.m = P.m;
    a.L = P.L;
    a.N = P.N;
    a.wstage = std::is_same<T, double>::value ? P.wstage
               : std::is_same<T, df32>::value ? P.wstage + kWinStageBytes / 16
                                              : nullptr;
    return a;
}

// Persistent grid of a kernel instance: SMs x resident CTAs per SM, set up
// once per instance (this also resolves the kernel on the device; the first
// plan creation does it for every instance before it queues any work).
static int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        NLH_CUDA(cudaGetDevice(&dev));
        NLH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

// Registers capped by launch bounds for more CTAs per SM (no spills in
// either): the FP32 2m = 8 default shape for 5 CTAs per SM (1% faster
// matvecs than the uncapped 4 CTAs), the FP32 2m = 12 default (3 x 2 teams,
// half lines) for 3 CTAs per SM (96 instead of 143 registers; 15% faster
// spreading on the 2048 x 2048 workload).
template <typename T, int W2, int NW, int TPB>
constexpr int spread_minb() {
    return (std::is_same<T, float>::value && W2 == 8 && NW == 1 && TPB == 4) ? 5
           : (std::is_same<T, float>::value && W2 == 12 && NW == 3 && TPB == 2) ? 3
                                                                               : 1;
}

template <typename T, int W2, int NW, int TPB, int SPLIT = 1>
static int spread_blocks() {
    static int blocks = 0;  // per template instance
    if (blocks == 0) {
        constexpr int NTH = 32 * NW * TPB;
        constexpr size_t smem = SpreadSmem<T, W2, NW, TPB>::bytes;
        auto kern = k_spread<T, W2, NW, TPB, spread_minb<T, W2, NW, TPB>(), SPLIT>;
        NLH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTH, smem));
        blocks = sm_count() * std::max(1, b);
    }
    return blocks;
}

template <typename T, int W2, int NW, int TPB, int SPLIT = 1>
static void launch_spread_shape(Plan &P, const double *x, typename Num<T>::G *grid,
                                const int *done, cudaStream_t s) {
    constexpr int NTH = 32 * NW * TPB;
    constexpr int MINB = spread_minb<T, W2, NW, TPB>();
    constexpr size_t smem = SpreadSmem<T, W2, NW, TPB>::bytes;
    auto kern = k_spread<T, W2, NW, TPB, MINB, SPLIT>;
    const int blocks = spread_blocks<T, W2, NW, TPB, SPLIT>();
    ProfRange pr(spread_class<T>(), s);
    // grid bound: the unit count once known on the host, else its upper bound
    const int64_t nu = P.n_units >= 0 ? P.n_units : P.units_cap;
    if (nu == 0) return;
    const unsigned g = (unsigned)std::min<int64_t>(blocks, nu);
    kern<<<g, NTH, smem, s>>>(nfft_args<T>(P), win_poly<T>(P), x, grid, done);
    NLH_CHECK_LAUNCH();
}

// Team shape (warps per team NW, teams per CTA TPB, x segments SPLIT) of the
// spreading kernel: fewer accumulators per thread (larger teams, split
// lines) against more independent teams per SM and fewer shared loads per
// multiply-add.  Shape 0 is the default; shapes 1 and 2 are compiled for the
// stencil widths of the workloads (2m = 8, 12).  The autotuner picks one per
// arithmetic (plan.team[]); other combinations run shape 0.  At 2m = 12
// every arithmetic splits its lines by default: 3-warp teams with 3 half
// lines per thread cover the 12 x 12 x 2 units without idle lanes (full
// lines on 2-warp teams leave a quarter of the team idle in its third
// pass); on the 2048 x 2048 workload this measured 11% faster for
// double-float and 8% for FP32.
template <typename T, int W2>
static void launch_spread(Plan &P, const double *x, typename Num<T>::G *grid, const int *done,
                          cudaStream_t s) {
    const int shape = P.team[arith_index<T>()];
    if constexpr (W2 == 8) {
        if (shape == 1) return launch_spread_shape<T, W2, 2, 2>(P, x, grid, done, s);
        if (shape == 2) return launch_spread_shape<T, W2, 2, 4>(P, x, grid, done, s);
    } else if constexpr (W2 == 12) {
        if (shape == 1) return launch_spread_shape<T, W2, 3, 4, 2>(P, x, grid, done, s);
        if (shape == 2) return launch_spread_shape<T, W2, 2, 2>(P, x, grid, done, s);
        return launch_spread_shape<T, W2, 3, 2, 2>(P, x, grid, done, s);
    }
    constexpr int NW = W2 <= 8 ? 1 : 2, TPB = W2 <= 8 ? 4 : 2;
    launch_spread_shape<T, W2, NW, TPB>(P, x, grid, done, s);
}

// Registers capped by launch bounds where that measured faster (no spills):
// double-float at 2m = 8 for 3 CTAs per SM, FP32 and double-float at 2m = 12
// for 2 CTAs per SM.
template <typename T, int W2>
constexpr int interp_minb() {
    return (std::is_same<T, df32>::value && W2 == 8) ? 3
           : (W2 == 12 && std::is_same<T, df32>::value) ? 2
                                                        : 1;
}
template <typename T, int W2>
constexpr size_t interp_smem() {
    return InterpTile<T, W2>::bytes + sizeof(int4) * kUnitItems + 16 + kWinStageBytes +
           (interp_smem_weights<T, W2>() ? 2 * W2 * sizeof(T) * interp_threads<T, W2>() : 0) +
           (interp_pairs<T, W2>() ? sizeof(int) * (kUnitItems + 1) : 0);
}

template <typename T, int W2>
static int interp_blocks() {
    static int blocks = 0;
    if (blocks == 0) {
        constexpr size_t smem = interp_smem<T, W2>();
        constexpr int NTH = interp_threads<T, W2>();
        auto kern = k_interp<T, W2, NTH, interp_minb<T, W2>()>;
        NLH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTH, smem));
        blocks = std::min(sm_count() * std::max(1, b), kPqSlots);
    }
    return blocks;
}

template <typename T, int W2>
static void launch_interp(Plan &P, const typename Num<T>::G *grid, const Epilogue &ep,
                          const int *done, cudaStream_t s) {
    constexpr int MINB = interp_minb<T, W2>();
    constexpr size_t smem = interp_smem<T, W2>();
    constexpr int NTH = interp_threads<T, W2>();
    auto kern = k_interp<T, W2, NTH, MINB>;
    const int blocks = interp_blocks<T, W2>();
    ProfRange pr(interp_class<T>(), s);
    const int64_t nu = P.n_units >= 0 ? P.n_units : P.units_cap;
    if (nu == 0) {
        NLH_REQUIRE(false, "internal: plan without work units");
    }
    const unsigned g = (unsigned)std::min<int64_t>(blocks, nu);
    kern<<<g, NTH, smem, s>>>(nfft_args<T>(P), win_poly<T>(P), grid, ep, done);
    NLH_CHECK_LAUNCH();
}

template <typename T, int W2>
static void spread_interp_w(Plan &P, bool spread, const double *x, typename Num<T>::G *grid,
                            const Epilogue *ep, const int *done, cudaStream_t s) {
    if (spread) launch_spread<T, W2>(P, x, grid, done, s);
    else launch_interp<T, W2>(P, grid, *ep, done, s);
}

template <typename T>
static void spread_interp(Plan &P, bool spread, const double *x, typename Num<T>::G *grid,
                          const Epilogue *ep, const int *done, cudaStream_t s) {
    switch (P.W2) {
        case 4: spread_interp_w<T, 4>(P, spread, x, grid, ep, done, s); break;
        case 6: spread_interp_w<T, 6>(P, spread, x, grid, ep, done, s); break;
        case 8: spread_interp_w<T, 8>(P, spread, x, grid, ep, done, s); break;
        case 10: spread_interp_w<T, 10>(P, spread, x, grid, ep, done, s); break;
        case 12: spread_interp_w<T, 12>(P, spread, x, grid, ep, done, s); break;
        case 14: spread_interp_w<T, 14>(P, spread, x, grid, ep, done, s); break;
        case 16: spread_interp_w<T, 16>(P, spread, x, grid, ep, done, s); break;
        default: NLH_REQUIRE(false, "internal: unsupported stencil width %d", P.W2);
    }
}

// Sets up (and thereby resolves on the device) every kernel instance of one
// arithmetic: the spreading shapes and the interpolation of every stencil
// width, and the convolution of every grid size.
template <typename T, int W2>
static void prepare_w() {
    if constexpr (W2 == 8) {
        spread_blocks<T, W2, 2, 2>();
        spread_blocks<T, W2, 2, 4>();
    } else if constexpr (W2 == 12) {
        spread_blocks<T, W2, 3, 4, 2>();
        spread_blocks<T, W2, 3, 2, 2>();
    }
    spread_blocks<T, W2, (W2 <= 8 ? 1 : 2), (W2 <= 8 ? 4 : 2)>();
    interp_blocks<T, W2>();
}

template <typename T>
static void prepare_t() {
    prepare_w<T, 4>();
    prepare_w<T, 6>();
    prepare_w<T, 8>();
    prepare_w<T, 10>();
    prepare_w<T, 12>();
    prepare_w<T, 14>();
    prepare_w<T, 16>();
    NLH_CUDA(cudaFuncSetAttribute(k_conv_xy<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)conv_xy_smem<T>(32)));
    NLH_CUDA(cudaFuncSetAttribute(k_conv_xy<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)conv_xy_smem<T>(64)));
    NLH_CUDA(cudaFuncSetAttribute(k_conv_xy<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)conv_xy_smem<T>(128)));
    cudaFuncAttributes fa;
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_conv<T, 1>));
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_conv<T, 2>));
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_conv<T, 4>));
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_conv<T, 8>));
}

template <typename T>
static void convolve(Plan &P, typename Num<T>::G *src, typename Num<T>::G *dst, const T *tab,
                     const typename Vec2<T>::type *tw, const int *done, cudaStream_t s) {
    const int n = P.n;
    dim3 gdim((unsigned)(n * n / 16), (unsigned)P.L);
    ProfRange pr(sizeof(T) == 4 ? NLH_K_CONV32 : NLH_K_CONV64, s);
    if (n <= 128) {  // x and y in one plane kernel, then z: 2 launches
        const size_t smem = conv_xy_smem<T>(n);
        const dim3 pdim((unsigned)n, (unsigned)P.L);
        switch (n) {
            case 32: k_conv_xy<T, 1><<<pdim, kConvXYThreads, smem, s>>>(src, dst, tab, tw, P.unit_ctr, done); break;
            case 64: k_conv_xy<T, 2><<<pdim, kConvXYThreads, smem, s>>>(src, dst, tab, tw, P.unit_ctr, done); break;
            default: k_conv_xy<T, 4><<<pdim, kConvXYThreads, smem, s>>>(src, dst, tab, tw, P.unit_ctr, done); break;
        }
        NLH_CHECK_LAUNCH();
        switch (n) {
            case 32: k_conv<T, 1><<<gdim, 256, 0, s>>>(dst, dst, 2, tab, tw, nullptr, done); break;
            case 64: k_conv<T, 2><<<gdim, 256, 0, s>>>(dst, dst, 2, tab, tw, nullptr, done); break;
            default: k_conv<T, 4><<<gdim, 256, 0, s>>>(dst, dst, 2, tab, tw, nullptr, done); break;
        }
        NLH_CHECK_LAUNCH();
        return;
    }
    for (int axis = 0; axis < 3; ++axis) {
        using G = typename Num<T>::G;
        G *in = axis == 0 ? src : dst;
        int *rst = axis == 0 ? P.unit_ctr : nullptr;
        switch (n) {
            case 32: k_conv<T, 1><<<gdim, 256, 0, s>>>(in, dst, axis, tab, tw, rst, done); break;
            case 64: k_conv<T, 2><<<gdim, 256, 0, s>>>(in, dst, axis, tab, tw, rst, done); break;
            case 128: k_conv<T, 4><<<gdim, 256, 0, s>>>(in, dst, axis, tab, tw, rst, done); break;
            case 256: k_conv<T, 8><<<gdim, 256, 0, s>>>(in, dst, axis, tab, tw, rst, done); break;
            default: NLH_REQUIRE(false, "internal: unsupported grid size %d", n);
        }
        NLH_CHECK_LAUNCH();
    }
}

__global__ void k_finish(double *__restrict__ yacc, const double *__restrict__ x,
                         const double *__restrict__ d, double *__restrict__ y, int64_t N,
                         double inv_l, int op, double alpha_val,
                         const double *__restrict__ alpha_dev, double *__restrict__ partials,
                         int nparts, const int *__restrict__ done);

// One matvec in arithmetic T: spread (with the gather of x), convolve the
// grids, interpolate with the epilogue.  Between matvecs the spread grids,
// the per-pixel sums and counts are zero and the unit counters are reset.
template <typename T>
static void matvec_t(Plan &P, int op, double alpha, const double *alpha_dev, const double *x,
                     double *y, double *partials, const int *done, typename Num<T>::G *gridA,
                     typename Num<T>::G *gridB, const T *tab, const typename Vec2<T>::type *tw,
                     const double *d, cudaStream_t s) {
    spread_interp<T>(P, true, x, gridA, nullptr, done, s);
    convolve<T>(P, gridA, gridB, tab, tw, done, s);
    Epilogue ep;
    ep.x = x;
    ep.d = d;
    ep.y = y;
    ep.yacc = P.yacc;
    ep.partials = partials;
    ep.nparts = kPqSlots;
    ep.L = P.L;
    ep.inv_l = 1.0 / P.L_norm;
    ep.op = op;
    ep.alpha = alpha;
    ep.alpha_dev = alpha_dev;
    spread_interp<T>(P, false, nullptr, gridB, &ep, done, s);
    if (P.L > 1) {
        ProfRange pr(NLH_K_EPILOGUE, s);
        k_finish<<<kRedBlocks, kRedThreads, 0, s>>>(P.yacc, x, d, y, P.N, ep.inv_l, op, alpha,
                                                    alpha_dev, partials, kPqSlots, done);
        NLH_CHECK_LAUNCH();
    }
}

// The epilogue of a plan that holds a range of the windows, after its share
// of Gamma_full x has been summed over the ranks into y: y = op(x, y) in place
// (as in the interpolation's epilogue) with the block partials of x^T y.
__global__ void __launch_bounds__(kRedThreads)
k_share_epilogue(const double *__restrict__ x, const double *__restrict__ d, double *__restrict__ y,
                 int64_t N, int op, double alpha_val, const double *__restrict__ alpha_dev,
                 double *__restrict__ partials, int nparts, const int *__restrict__ done) {
    __shared__ double sh[33];
    if (done && *done) return;
    const double alpha = alpha_dev ? *alpha_dev : alpha_val;
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double s = y[i], xi = x[i];
        double out = s;
        if (op != 0) {
            out = d[i] * xi - s;
            if (op == 2) out = fma(alpha, xi, out);
        }
        y[i] = out;
        part = fma(xi, out, part);
    }
    if (partials) {
        const double bs = block_sum(part, sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = bs;
        if (blockIdx.x == 0)
            for (int j = gridDim.x + threadIdx.x; j < nparts; j += blockDim.x) partials[j] = 0.0;
    }
}

// The epilogue of a plan of several windows, after every window has added
// its values into the per-pixel sums: y = op(x, inv_l sum) with the block
// partials of x^T y; the sums are cleared for the next matvec.
__global__ void __launch_bounds__(kRedThreads)
k_finish(double *__restrict__ yacc, const double *__restrict__ x, const double *__restrict__ d,
         double *__restrict__ y, int64_t N, double inv_l, int op, double alpha_val,
         const double *__restrict__ alpha_dev, double *__restrict__ partials, int nparts,
         const int *__restrict__ done) {
    __shared__ double sh[33];
    if (done && *done) return;
    const double alpha = alpha_dev ? *alpha_dev : alpha_val;
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double s = yacc[i] * inv_l;
        yacc[i] = 0.0;
        double out = s;
        if (op != 0) {
            const double xi = x[i];
            out = d[i] * xi - s;
            if (op == 2) out = fma(alpha, xi, out);
        }
        y[i] = out;
        if (partials) part = fma(x[i], out, part);
    }
    if (partials) {
        const double bs = block_sum(part, sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = bs;
        if (blockIdx.x == 0)
            for (int j = gridDim.x + threadIdx.x; j < nparts; j += blockDim.x) partials[j] = 0.0;
    }
}

static void matvec_prec(Plan &P, int op, int prec, double alpha, const double *x, double *y,
                        double *partials, const int *done, cudaStream_t s,
                        const double *alpha_dev) {
    if (prec == NLH_FP64) {
        NLH_REQUIRE(P.precision & 1, "matvec: FP64 path not built in this plan");
        matvec_t<double>(P, op, alpha, alpha_dev, x, y, partials, done, P.gridA64, P.gridB64,
                         P.tab64, P.tw64, P.d64, s);
    } else if (prec == NLH_FP32) {
        NLH_REQUIRE(P.precision & 2, "matvec: FP32 path not built in this plan");
        matvec_t<float>(P, op, alpha, alpha_dev, x, y, partials, done, P.gridA32, P.gridB32,
                        P.tab32, P.tw32, P.d32, s);
    } else {
        NLH_REQUIRE(P.precision & 4, "matvec: double-float path not built in this plan");
        matvec_t<df32>(P, op, alpha, alpha_dev, x, y, partials, done, P.gridA64, P.gridB64,
                       reinterpret_cast<const df32 *>(P.tabdf),
                       reinterpret_cast<const cdf *>(P.twdf), P.ddf, s);
    }
}

static const double *degrees_of(const Plan &P, int prec) {
    return prec == NLH_FP64 ? P.d64 : prec == NLH_FP32 ? P.d32 : P.ddf;
}

// A plan of all windows runs the matvec directly.  A plan that holds a range
// of the windows computes its share of Gamma_full x (normalised by the count
// of all windows); with a reduce callback that share is summed over the
// ranks in y and the epilogue follows, so that every op is the operator of
// all windows; without one, only op 0 (the share itself) is defined.
void matvec(Plan &P, int op, int prec, double alpha, const double *x, double *y,
            double *partials, const int *done, cudaStream_t s, const double *alpha_dev) {
    if (P.L == P.L_norm) {
        matvec_prec(P, op, prec, alpha, x, y, partials, done, s, alpha_dev);
        return;
    }
    NLH_REQUIRE(op == 0 || P.reduce_fn,
                "matvec: op %d on a plan of a window range needs a reduce callback", op);
    matvec_prec(P, 0, prec, 0.0, x, y, nullptr, done, s, nullptr);
    if (!P.reduce_fn) return;
    P.reduce_fn(y, P.N, (void *)s, P.reduce_ctx);
    if (op == 0 && !partials) return;
    ProfRange pr(NLH_K_EPILOGUE, s);
    k_share_epilogue<<<kRedBlocks, kRedThreads, 0, s>>>(x, degrees_of(P, prec), y, P.N, op, alpha,
                                                        alpha_dev, partials, kPqSlots, done);
    NLH_CHECK_LAUNCH();
}

// Resolves every NFFT kernel of the library on the current device once, so
// that no kernel is first loaded while a plan's work is queued or a solve is
// being captured.
void prepare_nfft_kernels() {
    static std::mutex mu;
    static bool done_once[64] = {false};
    int dev = 0;
    NLH_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done_once[dev]) return;
    prepare_t<double>();
    prepare_t<float>();
    prepare_t<df32>();
    cudaFuncAttributes fa;
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_share_epilogue));
    NLH_CUDA(cudaFuncGetAttributes(&fa, k_finish));
    if (dev >= 0 && dev < 64) done_once[dev] = true;
}

// Takes the first failed index check of the NFFT kernels (and clears the
// record); returns 0 if there was none.  Synchronous.
int nfft_check_take(int *info5) {
    int rec[5] = {0, 0, 0, 0, 0};
    NLH_CUDA(cudaMemcpyFromSymbol(rec, g_nfft_check, sizeof rec));
    if (rec[0] != 0) {
        const int zero[5] = {0, 0, 0, 0, 0};
        NLH_CUDA(cudaMemcpyToSymbol(g_nfft_check, zero, sizeof zero));
    }
    if (info5)
        for (int k = 0; k < 5; ++k) info5[k] = rec[k];
    return rec[0];
}

}  // namespace nlh

extern "C" nlh_status nlh_matvec(nlh_plan plan, int op, int precision, double alpha,
                                 const double *x, double *y, void *stream) {
    nlh::clear_error();
    try {
        NLH_REQUIRE(plan && x && y, "nlh_matvec: NULL pointer");
        NLH_REQUIRE(x != y, "nlh_matvec: x and y must not alias");
        NLH_REQUIRE(op >= 0 && op <= 2, "nlh_matvec: op=%d", op);
        NLH_REQUIRE(precision == NLH_FP64 || precision == NLH_FP32 || precision == NLH_DF32,
                    "nlh_matvec: precision=%d", precision);
        plan->stream = (cudaStream_t)stream;
        nlh::matvec(*plan, op, precision, alpha, x, y, nullptr, nullptr, (cudaStream_t)stream);
        return NLH_OK;
    } catch (nlh::Failure &f) {
        return f.st;
    }
}
