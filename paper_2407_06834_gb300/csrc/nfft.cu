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

#include <type_traits>
#include "async_copy.cuh"
#include "df32.cuh"

#include <algorithm>

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

constexpr int kChunk = 32;  // points staged in shared memory at a time

// Storage of one arithmetic: R = element of the weight records, G = grid
// element.  A weight record holds, per dim t, 2m values (R = T) or, for
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

// A team is NW warps; a CTA holds TPB teams.  Teams synchronise among
// themselves only (a warp sync, or a named barrier for two-warp teams).
template <int NW>
__device__ __forceinline__ void team_sync(int team) {
    if (NW == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(32 * NW) : "memory");
    }
}

// Weight record of one point: 3 x 2m values padded to a multiple of 16
// bytes so that a chunk of records is one bulk copy.
template <typename T, int W2>
constexpr int padded_record() {
    using R = typename Num<T>::R;
    return ((3 * Num<T>::kParts * W2 * (int)sizeof(R) + 15) / 16) * 16 / (int)sizeof(R);
}

constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared memory of one unit: the tile region (kTile + 2m - 1)^3, per team
// two staging buffers of kChunk weight records, two mbarriers, a status word
// and kChunk reduction slots.
template <typename T, int W2, int TPB>
struct UnitSmem {
    static constexpr int E = kTile + W2 - 1, E3 = E * E * E, PWP = padded_record<T, W2>();
    static constexpr size_t tile = align16(sizeof(T) * E3);
    static constexpr size_t stage = align16(sizeof(typename Num<T>::R) * kChunk * PWP);
    // per team: two staging buffers, two mbarriers, a status word and a slot,
    // and the per-warp point totals of a chunk (up to 4 warps per team)
    static constexpr size_t team = 2 * stage + 2 * sizeof(uint64_t) + 16 + align16(sizeof(T) * kChunk * 4);
};

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

template <int NW>
__device__ __forceinline__ ChunkCursor next_chunk(const ChunkCursor &c, const int4 *s_items,
                                                  int nit, int *s_next, int *s_slot, int team,
                                                  int tid) {
    ChunkCursor d = c;
    d.c0 += kChunk;
    if (d.c0 < d.cnt) return d;
    return make_cursor(s_items, fetch_item<NW>(s_next, s_slot, team, tid), nit);
}

// Per-team staging pipeline: thread 0 of the team issues the bulk copy of
// a chunk's weight records and waits for it (bounded); the team then reads.
template <typename T, int W2, int NW>
struct Stager {
    using R = typename Num<T>::R;
    static constexpr int PWP = padded_record<T, W2>();
    // two buffers, selected by b in {0, 1} without indexing an array (so the
    // state stays in registers)
    R *buf0, *buf1;
    uint64_t *bar;
    volatile int *flag;
    uint32_t phase0, phase1;
    bool pending0, pending1;
    int team, tid;

    __device__ __forceinline__ R *buf(int b) const { return b ? buf1 : buf0; }

    __device__ __forceinline__ void issue(int b, const R *wts, const ChunkCursor &c) {
        if (tid == 0) {
            const int cn = min(kChunk, c.cnt - c.c0);
            const uint32_t bytes = (uint32_t)(cn * PWP * sizeof(R));
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[b], bytes);
            bulk_copy_g2s(buf(b), wts + (int64_t)(c.start + c.c0) * PWP, bytes, &bar[b]);
        }
        if (b) pending1 = true; else pending0 = true;
    }

    // Returns false if the copy timed out (the team then stops).
    __device__ __forceinline__ bool wait(int b, int *err) {
        const uint32_t ph = b ? phase1 : phase0;
        if (tid == 0) *flag = mbar_wait_bounded(&bar[b], ph, err) ? 1 : 0;
        team_sync<NW>(team);
        bool ok = *flag != 0;
        if (ok) ok = mbar_try_wait(&bar[b], ph);  // acquire for every reader
        if (b) { phase1 ^= 1u; pending1 = false; } else { phase0 ^= 1u; pending0 = false; }
        return ok;
    }

    // On an early exit: wait (bounded) for copies still in flight.
    __device__ __forceinline__ void drain(int *err) {
        if (tid != 0) return;
        if (pending0) mbar_wait_bounded(&bar[0], phase0, err);
        if (pending1) mbar_wait_bounded(&bar[1], phase1, err);
    }
};

// Team area: two staging buffers, two mbarriers, a status word, a
// broadcast slot, kChunk reduction values.
template <typename T, int W2, int NW, int TPB>
__device__ __forceinline__ Stager<T, W2, NW> make_stager(unsigned char *team_base, int team,
                                                         int tid) {
    using SM = UnitSmem<T, W2, TPB>;
    Stager<T, W2, NW> st;
    st.buf0 = reinterpret_cast<typename Num<T>::R *>(team_base);
    st.buf1 = reinterpret_cast<typename Num<T>::R *>(team_base + SM::stage);
    st.bar = reinterpret_cast<uint64_t *>(team_base + 2 * SM::stage);
    st.flag = reinterpret_cast<volatile int *>(team_base + 2 * SM::stage + 2 * sizeof(uint64_t));
    st.phase0 = st.phase1 = 0u;
    st.pending0 = st.pending1 = false;
    st.team = team;
    st.tid = tid;
    return st;
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
    __device__ __forceinline__ void set(int a, T x) { v[a] = x; }
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
    __device__ __forceinline__ void axpy(float s, const Line &w) {
        unsigned long long ss;
        asm("mov.b64 %0, {%1, %1};" : "=l"(ss) : "f"(s));
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
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc));
        return lo + hi;
    }
    __device__ __forceinline__ float get(int a) const {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v[a / 2]));
        return (a & 1) ? hi : lo;
    }
    __device__ __forceinline__ void set(int a, float x) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v[a / 2]));
        if (a & 1) hi = x; else lo = x;
        asm("mov.b64 %0, {%1, %2};" : "=l"(v[a / 2]) : "f"(lo), "f"(hi));
    }
    __device__ __forceinline__ void load_cells(const float *row) {  // 2m consecutive cells
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a)
            asm("mov.b64 %0, {%1, %2};" : "=l"(v[a]) : "f"(row[2 * a]), "f"(row[2 * a + 1]));
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
    __device__ __forceinline__ void load(const float *src) {
#pragma unroll
        for (int a = 0; a < W2 / 2; ++a) {
            h[a] = reinterpret_cast<const unsigned long long *>(src)[a];
            l[a] = reinterpret_cast<const unsigned long long *>(src + W2)[a];
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
    __device__ __forceinline__ void set(int a, df32 x) {
        float h0, h1, l0, l1;
        pk_split(h[a / 2], h0, h1);
        pk_split(l[a / 2], l0, l1);
        if (a & 1) { h1 = x.hi; l1 = x.lo; } else { h0 = x.hi; l0 = x.lo; }
        h[a / 2] = pk_make(h0, h1);
        l[a / 2] = pk_make(l0, l1);
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

// (y, z) stencil pairs owned by one thread: pair p = tid + NT k.  When the
// team size is a multiple of 2m every pair of a thread has the same y offset.
template <int W2, int NT, int PPT>
struct Pairs {
    int b0, bb[PPT], cc[PPT];
    bool ok[PPT];
    static constexpr bool kSameB = (NT % W2) == 0;
    __device__ __forceinline__ void init(int tid) {
        b0 = tid % W2;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            int p = tid + NT * k;
            ok[k] = p < W2 * W2;
            bb[k] = kSameB ? b0 : (ok[k] ? p % W2 : 0);
            cc[k] = ok[k] ? p / W2 : 0;
        }
    }
};

// Shared carve-up common to both kernels: tile region, item records, the
// CTA's item counter, then TPB team areas.
template <typename T, int W2, int TPB>
struct UnitLayout {
    using SM = UnitSmem<T, W2, TPB>;
    static constexpr size_t items_off = SM::tile;
    static constexpr size_t next_off = items_off + sizeof(int4) * kUnitItems;  // 4 ints:
    // [0] item counter, [1] current unit, [2] abort flag
    static constexpr size_t teams_off = next_off + 16;
    static constexpr size_t bytes = teams_off + TPB * SM::team;
};

// ------------------------------------------------------------------ spreading
// Persistent CTAs take units from a global counter (units are stored in
// decreasing size).  Per unit, each team takes items; a thread owns PPT
// (y, z) stencil pairs with their full x line of 2m accumulators, summed in
// registers over the item's points (all points of an item share the
// stencil).  Items are then added into the shared tile, and the tile is
// added into the global grid once (non-zero entries only).  xs holds the
// input vector in sorted order.
template <typename T, int W2, int NW, int TPB, int MINB = 1>
__global__ void __launch_bounds__(32 * NW * TPB, MINB)
k_spread(const int4 *__restrict__ units, const int *__restrict__ n_units_dev,
         int *__restrict__ unit_ctr,
         const int4 *__restrict__ items, const typename Num<T>::R *__restrict__ wts,
         const T *__restrict__ xs, typename Num<T>::G *__restrict__ grid, int n, int m,
         const int *__restrict__ done, int *__restrict__ err) {
    using R = typename Num<T>::R;
    using G = typename Num<T>::G;
    using SM = UnitSmem<T, W2, TPB>;
    using LY = UnitLayout<T, W2, TPB>;
    constexpr int NT = 32 * NW, PPT = (W2 * W2 + NT - 1) / NT, PWP = SM::PWP;
    constexpr int E = SM::E, E3 = SM::E3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + LY::items_off);
    int *s_ctl = reinterpret_cast<int *>(smem_raw + LY::next_off);
    if (done && *done) return;
    const int team = threadIdx.x / NT, tid = threadIdx.x % NT, lane = tid & 31;
    unsigned char *team_base = smem_raw + LY::teams_off + team * SM::team;
    auto st = make_stager<T, W2, NW, TPB>(team_base, team, tid);
    int *s_slot = const_cast<int *>(st.flag) + 1;
    if (tid == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_ctl[2] = 0;
    Pairs<W2, NT, PPT> pr;
    pr.init(tid);
    const int msk = n - 1;
    while (true) {
        __syncthreads();  // previous unit fully flushed
        if (threadIdx.x == 0) s_ctl[1] = atomicAdd(unit_ctr, 1);
        __syncthreads();
        const int uidx = s_ctl[1];
        if (uidx >= *n_units_dev || s_ctl[2]) break;
        const int4 un = units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        int tx0, ty0, tz0;
        tile_origin(un.y, n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < E3; e += blockDim.x) S[e] = T(0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = items[it0 + e];
        if (threadIdx.x == 0) s_ctl[0] = TPB;
        __syncthreads();
        Line<T, W2> acc[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[k].zero();
        ChunkCursor cur = make_cursor(s_items, team, nit);
        T vcur = T(0);
        if (cur.valid()) {
            st.issue(0, wts, cur);
            if (lane < cur.cnt) vcur = xs[cur.start + lane];
        }
        int bsel = 0;
        while (cur.valid()) {
            const ChunkCursor nxt = next_chunk<NW>(cur, s_items, nit, s_ctl, s_slot, team, tid);
            T vnxt = T(0);
            if (nxt.valid()) {
                st.issue(bsel ^ 1, wts, nxt);
                if (lane < nxt.cnt - nxt.c0) vnxt = xs[nxt.start + nxt.c0 + lane];
            }
            if (!st.wait(bsel, err)) {
                st.drain(err);
                s_ctl[2] = 1;
                break;
            }
            const R *sw = st.buf(bsel);
            const int cn = min(kChunk, cur.cnt - cur.c0);
            for (int j = 0; j < cn; ++j) {
                const R *wp = sw + j * PWP;
                Line<T, W2> wx;
                wx.load(rec_line<T, W2>(wp, 0));
                const T vj = __shfl_sync(0xffffffffu, vcur, j);
                if (Pairs<W2, NT, PPT>::kSameB) {
                    const T vb = vj * rec_val<T, W2>(wp, 1, pr.b0);
#pragma unroll
                    for (int k = 0; k < PPT; ++k)
                        if (pr.ok[k]) acc[k].axpy(vb * rec_val<T, W2>(wp, 2, pr.cc[k]), wx);
                } else {
#pragma unroll
                    for (int k = 0; k < PPT; ++k)
                        if (pr.ok[k])
                            acc[k].axpy(vj * rec_val<T, W2>(wp, 1, pr.bb[k]) *
                                            rec_val<T, W2>(wp, 2, pr.cc[k]),
                                        wx);
                }
            }
            if (cur.c0 + kChunk >= cur.cnt) {  // last chunk of the item: add into the tile
                int lx0, ly0, lz0;
                item_local(cur.local, lx0, ly0, lz0);
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (pr.ok[k]) {
                        T *row = S + ((lz0 + pr.cc[k]) * E + (ly0 + pr.bb[k])) * E + lx0;
#pragma unroll
                        for (int a = 0; a < W2; ++a) atomicAdd(&row[a], acc[k].get(a));
                    }
                    acc[k].zero();
                }
            }
            team_sync<NW>(team);  // every read of buffer bsel is done before it is refilled
            cur = nxt;
            vcur = vnxt;
            bsel ^= 1;
        }
        __syncthreads();
        G *g = grid + (int64_t)l * n * n * n;
        for (int e = threadIdx.x; e < E3; e += blockDim.x) {
            T val = S[e];
            if (val != T(0)) {
                int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
                int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                    gz = (tz0 - m + 1 + ez) & msk;
                atomicAdd(&g[((int64_t)gz * n + gy) * n + gx], (G)val);
            }
        }
    }
}

// ------------------------------------------------------------------ interpolation
// Persistent CTAs over units as in k_spread.  The tile region of the
// convolved grid is staged in shared memory; each team holds an item's
// stencil in registers and sums every point's 2m^3 products.  The
// per-thread partial sums of a chunk of 32 points are reduce-scattered over
// the warp so that lane j ends with point j's value.
template <typename T, int W2, int NW, int TPB>
__global__ void __launch_bounds__(32 * NW * TPB, 1)
k_interp(const int4 *__restrict__ units, const int *__restrict__ n_units_dev,
         int *__restrict__ unit_ctr,
         const int4 *__restrict__ items, const int *__restrict__ perm,
         const typename Num<T>::R *__restrict__ wts, const typename Num<T>::G *__restrict__ grid,
         double *__restrict__ Y, int n, int m, int64_t N, const int *__restrict__ done,
         int *__restrict__ err) {
    using R = typename Num<T>::R;
    using G = typename Num<T>::G;
    using SM = UnitSmem<T, W2, TPB>;
    using LY = UnitLayout<T, W2, TPB>;
    constexpr int NT = 32 * NW, PPT = (W2 * W2 + NT - 1) / NT, PWP = SM::PWP;
    constexpr int E = SM::E, E3 = SM::E3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + LY::items_off);
    int *s_ctl = reinterpret_cast<int *>(smem_raw + LY::next_off);
    if (done && *done) return;
    const int team = threadIdx.x / NT, tid = threadIdx.x % NT, lane = tid & 31, warp = tid >> 5;
    unsigned char *team_base = smem_raw + LY::teams_off + team * SM::team;
    auto st = make_stager<T, W2, NW, TPB>(team_base, team, tid);
    int *s_slot = const_cast<int *>(st.flag) + 1;
    T *sred = reinterpret_cast<T *>(team_base + 2 * SM::stage + 2 * sizeof(uint64_t) + 16);
    if (tid == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_ctl[2] = 0;
    Pairs<W2, NT, PPT> pr;
    pr.init(tid);
    const int msk = n - 1;
    while (true) {
        __syncthreads();  // previous unit done with the tile
        if (threadIdx.x == 0) s_ctl[1] = atomicAdd(unit_ctr, 1);
        __syncthreads();
        const int uidx = s_ctl[1];
        if (uidx >= *n_units_dev || s_ctl[2]) break;
        const int4 un = units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        int tx0, ty0, tz0;
        tile_origin(un.y, n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = items[it0 + e];
        if (threadIdx.x == 0) s_ctl[0] = TPB;
        const G *g = grid + (int64_t)l * n * n * n;
        {
            constexpr int UNR = 8;
            for (int base = threadIdx.x; base < E3; base += blockDim.x * UNR) {
                G vals[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    int e = base + u * blockDim.x;
                    vals[u] = G(0);
                    if (e < E3) {
                        int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
                        int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                            gz = (tz0 - m + 1 + ez) & msk;
                        vals[u] = __ldg(&g[((int64_t)gz * n + gy) * n + gx]);
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    int e = base + u * blockDim.x;
                    if (e < E3) S[e] = T(vals[u]);
                }
            }
        }
        __syncthreads();
        ChunkCursor cur = make_cursor(s_items, team, nit);
        if (cur.valid()) st.issue(0, wts, cur);
        int pcur = (cur.valid() && lane < cur.cnt) ? perm[cur.start + lane] : 0;
        Line<T, W2> H[PPT];
        int bsel = 0;
        while (cur.valid()) {
            if (cur.c0 == 0) {  // first chunk of an item: its stencil from the tile
                int lx0, ly0, lz0;
                item_local(cur.local, lx0, ly0, lz0);
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const T *row = S + ((lz0 + pr.cc[k]) * E + (ly0 + pr.bb[k])) * E + lx0;
#pragma unroll
                    for (int a = 0; a < W2; ++a) H[k].set(a, pr.ok[k] ? row[a] : T(0));
                }
            }
            const ChunkCursor nxt = next_chunk<NW>(cur, s_items, nit, s_ctl, s_slot, team, tid);
            int pnxt = 0;
            if (nxt.valid()) {
                st.issue(bsel ^ 1, wts, nxt);
                if (lane < nxt.cnt - nxt.c0) pnxt = perm[nxt.start + nxt.c0 + lane];
            }
            if (!st.wait(bsel, err)) {
                st.drain(err);
                s_ctl[2] = 1;
                break;
            }
            const R *sw = st.buf(bsel);
            const int cn = min(kChunk, cur.cnt - cur.c0);
            // Points in groups of 8: each thread forms its partial sums for the
            // group, an 8-lane reduce-scatter leaves lane l with the partial of
            // point (l & 7) over its 8-lane group, and two shuffle-adds finish the
            // warp sum.  A runtime loop over groups keeps the code small.
            for (int g0 = 0; g0 < cn; g0 += 8) {
                T part[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    T sum = T(0);
                    const int j = g0 + jj;
                    if (j < cn) {
                        const R *wp = sw + j * PWP;
                        Line<T, W2> wx;
                        wx.load(rec_line<T, W2>(wp, 0));
                        if (Pairs<W2, NT, PPT>::kSameB) {
                            T zs = T(0);
#pragma unroll
                            for (int k = 0; k < PPT; ++k)
                                if (pr.ok[k])
                                    zs = fma(rec_val<T, W2>(wp, 2, pr.cc[k]), wx.dot(H[k]), zs);
                            sum = rec_val<T, W2>(wp, 1, pr.b0) * zs;
                        } else {
#pragma unroll
                            for (int k = 0; k < PPT; ++k)
                                if (pr.ok[k])
                                    sum = fma(rec_val<T, W2>(wp, 1, pr.bb[k]) *
                                                  rec_val<T, W2>(wp, 2, pr.cc[k]),
                                              wx.dot(H[k]), sum);
                        }
                    }
                    part[jj] = sum;
                }
#pragma unroll
                for (int o = 4; o >= 1; o >>= 1) {
                    const bool upper = lane & o;
#pragma unroll
                    for (int kk = 0; kk < o; ++kk) {
                        T send = upper ? part[kk] : part[kk + o];
                        T keep = upper ? part[kk + o] : part[kk];
                        part[kk] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                T tot = part[0];
                tot = tot + __shfl_xor_sync(0xffffffffu, tot, 8);
                tot = tot + __shfl_xor_sync(0xffffffffu, tot, 16);
                if (NW > 1) {
                    // each warp's totals of the chunk's points; summed once per chunk
                    if (lane < 8) sred[warp * kChunk + g0 + lane] = tot;
                } else {
                    const int pidx = __shfl_sync(0xffffffffu, pcur, (g0 + lane) & 31);
                    if (lane < 8 && g0 + lane < cn) Y[(int64_t)l * N + pidx] = (double)tot;
                }
            }
            if (NW > 1) {
                team_sync<NW>(team);
                if (warp == 0 && lane < cn) {  // lane j holds point j's permutation entry
                    T tot = sred[lane];
#pragma unroll
                    for (int w = 1; w < NW; ++w) tot = tot + sred[w * kChunk + lane];
                    Y[(int64_t)l * N + pcur] = (double)tot;
                }
            }
            team_sync<NW>(team);  // every read of buffer bsel (and sred) is done
            cur = nxt;
            pcur = pnxt;
            bsel ^= 1;
        }
    }
}

template <typename T> constexpr int interp_class() {
    return sizeof(T) == 4 ? NLH_K_INTERP32 : (Num<T>::kParts == 2 ? NLH_K_INTERPDF : NLH_K_INTERP64);
}
template <typename T> constexpr int interp_class_pl() { return interp_class<T>(); }

// ------------------------------------------------- interpolation, points on lanes
// The same interpolation with one point per lane: a warp takes 32
// consecutive (sorted) points of the unit, each lane finds its point's cell
// among the unit's items (binary search on the first sorted positions),
// holds its weight record in registers and evaluates
//   y = sum_z wz[z] (wx . t_z),  t_z[x] = sum_y wy[y] S[z][y][x]
// over its stencil in the staged tile region, with no cross-lane reduction
// (consecutive points mostly share a cell, so their tile rows are the same
// addresses).  Written straight to Y in pixel order.
constexpr int kPlThreads = 256;

template <typename T, int W2, int NTH = kPlThreads, int MINB = 1>
__global__ void __launch_bounds__(NTH, MINB)
k_interp_pl(const int4 *__restrict__ units, const int *__restrict__ n_units_dev,
            int *__restrict__ unit_ctr, const int4 *__restrict__ items,
            const int *__restrict__ perm, const typename Num<T>::R *__restrict__ wts,
            const typename Num<T>::G *__restrict__ grid, double *__restrict__ Y, int n, int m,
            int64_t N, const int *__restrict__ done) {
    using R = typename Num<T>::R;
    using G = typename Num<T>::G;
    using SM = UnitSmem<T, W2, 1>;
    constexpr int E = SM::E, E3 = SM::E3, PWP = SM::PWP;
    static_assert((PWP * sizeof(R)) % 16 == 0, "records are whole 16-byte words");
    constexpr int RW = PWP * (int)sizeof(R) / 16;  // 16-byte words per record
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + SM::tile);
    int *s_ctl = reinterpret_cast<int *>(s_items + kUnitItems);
    if (done && *done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int msk = n - 1;
    while (true) {
        __syncthreads();  // previous unit done with the tile
        if (threadIdx.x == 0) s_ctl[0] = atomicAdd(unit_ctr, 1);
        __syncthreads();
        const int uidx = s_ctl[0];
        if (uidx >= *n_units_dev) break;
        const int4 un = units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        int tx0, ty0, tz0;
        tile_origin(un.y, n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = items[it0 + e];
        const G *g = grid + (int64_t)l * n * n * n;
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
                        vals[u] = __ldg(&g[((int64_t)gz * n + gy) * n + gx]);
                    }
                }
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int e = base + u * blockDim.x;
                    if (e < E3) S[e] = T(vals[u]);
                }
            }
        }
        __syncthreads();
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
            R rec[PWP];
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(wts + (int64_t)sp * PWP);
#pragma unroll
                for (int k = 0; k < RW; ++k) reinterpret_cast<uint4 *>(rec)[k] = __ldg(src + k);
            }
            Line<T, W2> wx, t, h;
            wx.load(rec_line<T, W2>(rec, 0));
            T wy[W2], wz[W2];
#pragma unroll
            for (int j = 0; j < W2; ++j) {
                wy[j] = rec_val<T, W2>(rec, 1, j);
                wz[j] = rec_val<T, W2>(rec, 2, j);
            }
            T acc = T(0);
            // the z loop stays rolled (the unrolled y loop is the work; a
            // fully unrolled stencil made the compile many minutes long)
#pragma unroll 1
            for (int z = 0; z < W2; ++z) {
                t.zero();
                const T *srow = S + ((lz0 + z) * E + ly0) * E + lx0;
#pragma unroll
                for (int y = 0; y < W2; ++y) {
                    h.load_cells(srow + y * E);
                    t.axpy(wy[y], h);
                }
                acc = fma(wz[z], wx.dot(t), acc);
            }
            Y[(int64_t)l * N + perm[sp]] = (double)acc;
        }
    }
}

template <typename T, int W2, int NTH, int MINB = 1>
static void launch_interp_pl_n(Plan &P, const typename Num<T>::R *wts, typename Num<T>::G *grid,
                               const int *done, cudaStream_t s) {
    constexpr size_t smem = UnitSmem<T, W2, 1>::tile + sizeof(int4) * kUnitItems + 16;
    if (P.units_cap == 0) return;
    static int blocks = 0;
    if (blocks == 0) {
        NLH_CUDA(cudaFuncSetAttribute(k_interp_pl<T, W2, NTH, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0, b = 0;
        NLH_CUDA(cudaGetDevice(&dev));
        NLH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_interp_pl<T, W2, NTH, MINB>, NTH,
                                                               smem));
        blocks = sms * std::max(1, b);
    }
    ProfRange pr(interp_class_pl<T>(), s);
    const int64_t nu = P.n_units >= 0 ? P.n_units : P.units_cap;
    if (nu == 0) return;
    const unsigned g = (unsigned)std::min<int64_t>(blocks, nu);
    k_interp_pl<T, W2, NTH, MINB><<<g, NTH, smem, s>>>(P.units, P.d_units, P.unit_ctr + 1, P.items,
                                                 P.perm, wts, grid, P.Y, P.n, P.m, P.N, done);
    NLH_CHECK_LAUNCH();
}

// 256 threads per CTA measured best for the double-float kernel at 512^2
// (0.286 ms against 0.340 ms with 128 and 0.353 ms with 512, uncapped).
template <typename T, int W2>
static void launch_interp_pl(Plan &P, const typename Num<T>::R *wts, typename Num<T>::G *grid,
                             const int *done, cudaStream_t s) {
    // Registers capped by launch bounds (no spills in any instance):
    //  double-float, 2m = 8: 3 CTAs per SM instead of 2 (whole matvecs at
    //    512^2 0.722 -> 0.627 ms);
    //  FP32 and double-float, 2m = 12: 2 CTAs per SM instead of 1 (whole
    //    matvecs at 2048^2, 5x5 patches: 20.75 -> 17.97 ms and 81.4 -> 75.0 ms).
    constexpr bool f64 = std::is_same<T, double>::value;
    constexpr int MINB = (std::is_same<T, df32>::value && W2 == 8) ? 3 : (W2 == 12 && !f64) ? 2 : 1;
    launch_interp_pl_n<T, W2, kPlThreads, MINB>(P, wts, grid, done, s);
}

// ------------------------------------------------------------------ tensor-core FP32 path
// For 2m = 8 the FP32 stencil work of one item (one grid cell, P points) is a
// dense contraction over a 64 x 8 block of the grid (rows (z, y), columns x):
//   spread:  G[(z,y), x] += sum_p (v_p wz_p[z] wy_p[y]) wx_p[x]   (A: 64 x P, B: P x 8)
//   interp:  C[(z,y), p]  = sum_x G[(z,y), x] wx_p[x],  y_p = sum wz wy C   (A: 64 x 8)
// These kernels run it on the tensor cores with mma.sync m16n8k8 TF32 and
// the 3xTF32 split (a = a_hi + a_lo, products hi*hi + hi*lo + lo*hi), which
// keeps FP32 accuracy (~2^-22 relative per product, FP32 accumulation).
// Rows are ordered so that m16 tile i holds z = 2i (rows 0-7) and z = 2i+1
// (rows 8-15) with y = row % 8; a thread (group g = lane / 4) then owns
// y = g and every z of its columns.
__device__ __forceinline__ uint32_t tf32_hi(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}
// a = hi + lo: hi keeps the top 10 mantissa bits (exact in TF32; a - hi is
// then exact in FP32), lo is that remainder rounded to TF32.
__device__ __forceinline__ void tf32_split(float a, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(a) & 0xFFFFE000u;
    lo = tf32_hi(a - __uint_as_float(hi));
}
// D += A B (m16n8k8, tf32 inputs, f32 accumulators)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// 3xTF32: D += Ahi Bhi + Ahi Blo + Alo Bhi
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4],
                                           const uint32_t (&al)[4], uint32_t bh0, uint32_t bh1,
                                           uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

template <int TPB, int MINB>
__global__ void __launch_bounds__(32 * TPB, MINB)
k_spread_tc(const int4 *__restrict__ units, const int *__restrict__ n_units_dev,
            int *__restrict__ unit_ctr, const int4 *__restrict__ items,
            const float *__restrict__ wts, const float *__restrict__ xs, float *__restrict__ grid,
            int n, int m, const int *__restrict__ done, int *__restrict__ err) {
    constexpr int W2 = 8, NW = 1;
    using SM = UnitSmem<float, W2, TPB>;
    using LY = UnitLayout<float, W2, TPB>;
    constexpr int PWP = SM::PWP, E = SM::E, E3 = SM::E3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *S = reinterpret_cast<float *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + LY::items_off);
    int *s_ctl = reinterpret_cast<int *>(smem_raw + LY::next_off);
    if (done && *done) return;
    const int team = threadIdx.x / 32, lane = threadIdx.x % 32, tid = lane;
    const int g = lane >> 2, t = lane & 3;
    unsigned char *team_base = smem_raw + LY::teams_off + team * SM::team;
    auto st = make_stager<float, W2, NW, TPB>(team_base, team, tid);
    int *s_slot = const_cast<int *>(st.flag) + 1;
    if (tid == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_ctl[2] = 0;
    const int msk = n - 1;
    while (true) {
        __syncthreads();  // previous unit fully flushed
        if (threadIdx.x == 0) s_ctl[1] = atomicAdd(unit_ctr, 1);
        __syncthreads();
        const int uidx = s_ctl[1];
        if (uidx >= *n_units_dev || s_ctl[2]) break;
        const int4 un = units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        int tx0, ty0, tz0;
        tile_origin(un.y, n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < E3; e += blockDim.x) S[e] = 0.f;
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = items[it0 + e];
        if (threadIdx.x == 0) s_ctl[0] = TPB;
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][e] = 0.f;
        ChunkCursor cur = make_cursor(s_items, team, nit);
        float vcur = 0.f;
        if (cur.valid()) {
            st.issue(0, wts, cur);
            if (lane < cur.cnt) vcur = xs[cur.start + lane];
        }
        int bsel = 0;
        while (cur.valid()) {
            const ChunkCursor nxt = next_chunk<NW>(cur, s_items, nit, s_ctl, s_slot, team, tid);
            float vnxt = 0.f;
            if (nxt.valid()) {
                st.issue(bsel ^ 1, wts, nxt);
                if (lane < nxt.cnt - nxt.c0) vnxt = xs[nxt.start + nxt.c0 + lane];
            }
            if (!st.wait(bsel, err)) {
                st.drain(err);
                s_ctl[2] = 1;
                break;
            }
            const float *sw = st.buf(bsel);
            const int cn = min(kChunk, cur.cnt - cur.c0);
            for (int g0 = 0; g0 < cn; g0 += 8) {
                // columns t and t + 4 of this 8-point group
                const int p0 = g0 + t, p1 = g0 + t + 4;
                const float v0 = __shfl_sync(0xffffffffu, vcur, p0);
                const float v1 = __shfl_sync(0xffffffffu, vcur, p1 & 31);
                const bool ok0 = p0 < cn, ok1 = p1 < cn;
                const float *w0 = sw + p0 * PWP, *w1 = sw + (ok1 ? p1 : p0) * PWP;
                const float s0 = ok0 ? v0 * w0[W2 + g] : 0.f;
                const float s1 = ok1 ? v1 * w1[W2 + g] : 0.f;
                // columns of points past the chunk are zero (the staging buffer
                // beyond cn holds stale records)
                const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 z0a = ok0 ? *reinterpret_cast<const float4 *>(w0 + 2 * W2) : zero4;
                const float4 z0b = ok0 ? *reinterpret_cast<const float4 *>(w0 + 2 * W2 + 4) : zero4;
                const float4 z1a = ok1 ? *reinterpret_cast<const float4 *>(w1 + 2 * W2) : zero4;
                const float4 z1b = ok1 ? *reinterpret_cast<const float4 *>(w1 + 2 * W2 + 4) : zero4;
                const float wz0[8] = {z0a.x, z0a.y, z0a.z, z0a.w, z0b.x, z0b.y, z0b.z, z0b.w};
                const float wz1[8] = {z1a.x, z1a.y, z1a.z, z1a.w, z1b.x, z1b.y, z1b.z, z1b.w};
                // B: k = point (t, t + 4), n = x = g
                uint32_t bh0, bl0, bh1, bl1;
                tf32_split(ok0 ? w0[g] : 0.f, bh0, bl0);
                tf32_split(ok1 ? w1[g] : 0.f, bh1, bl1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint32_t ah[4], al[4];
                    tf32_split(s0 * wz0[2 * i], ah[0], al[0]);
                    tf32_split(s0 * wz0[2 * i + 1], ah[1], al[1]);
                    tf32_split(s1 * wz1[2 * i], ah[2], al[2]);
                    tf32_split(s1 * wz1[2 * i + 1], ah[3], al[3]);
                    mma_3xtf32(acc[i], ah, al, bh0, bh1, bl0, bl1);
                }
            }
            if (cur.c0 + kChunk >= cur.cnt) {  // last chunk of the item: add into the tile
                int lx0, ly0, lz0;
                item_local(cur.local, lx0, ly0, lz0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float *row = S + ((lz0 + 2 * i + h) * E + (ly0 + g)) * E + lx0 + 2 * t;
                        atomicAdd(&row[0], acc[i][2 * h]);
                        atomicAdd(&row[1], acc[i][2 * h + 1]);
                        acc[i][2 * h] = acc[i][2 * h + 1] = 0.f;
                    }
                }
            }
            __syncwarp();  // every read of buffer bsel is done before it is refilled
            cur = nxt;
            vcur = vnxt;
            bsel ^= 1;
        }
        __syncthreads();
        float *gl = grid + (int64_t)l * n * n * n;
        for (int e = threadIdx.x; e < E3; e += blockDim.x) {
            const float val = S[e];
            if (val != 0.f) {
                int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
                int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                    gz = (tz0 - m + 1 + ez) & msk;
                atomicAdd(&gl[((int64_t)gz * n + gy) * n + gx], val);
            }
        }
    }
}

template <int TPB, int MINB>
__global__ void __launch_bounds__(32 * TPB, MINB)
k_interp_tc(const int4 *__restrict__ units, const int *__restrict__ n_units_dev,
            int *__restrict__ unit_ctr, const int4 *__restrict__ items,
            const int *__restrict__ perm, const float *__restrict__ wts,
            const float *__restrict__ grid, double *__restrict__ Y, int n, int m, int64_t N,
            const int *__restrict__ done, int *__restrict__ err) {
    constexpr int W2 = 8, NW = 1;
    using SM = UnitSmem<float, W2, TPB>;
    using LY = UnitLayout<float, W2, TPB>;
    constexpr int PWP = SM::PWP, E = SM::E, E3 = SM::E3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *S = reinterpret_cast<float *>(smem_raw);
    int4 *s_items = reinterpret_cast<int4 *>(smem_raw + LY::items_off);
    int *s_ctl = reinterpret_cast<int *>(smem_raw + LY::next_off);
    if (done && *done) return;
    const int team = threadIdx.x / 32, lane = threadIdx.x % 32, tid = lane;
    const int g = lane >> 2, t = lane & 3;
    unsigned char *team_base = smem_raw + LY::teams_off + team * SM::team;
    auto st = make_stager<float, W2, NW, TPB>(team_base, team, tid);
    int *s_slot = const_cast<int *>(st.flag) + 1;
    if (tid == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_ctl[2] = 0;
    const int msk = n - 1;
    while (true) {
        __syncthreads();  // previous unit done with the tile
        if (threadIdx.x == 0) s_ctl[1] = atomicAdd(unit_ctr, 1);
        __syncthreads();
        const int uidx = s_ctl[1];
        if (uidx >= *n_units_dev || s_ctl[2]) break;
        const int4 un = units[uidx];
        const int l = un.x, it0 = un.z, nit = un.w;
        int tx0, ty0, tz0;
        tile_origin(un.y, n, tx0, ty0, tz0);
        for (int e = threadIdx.x; e < nit; e += blockDim.x) s_items[e] = items[it0 + e];
        if (threadIdx.x == 0) s_ctl[0] = TPB;
        const float *gl = grid + (int64_t)l * n * n * n;
        for (int e = threadIdx.x; e < E3; e += blockDim.x) {
            int ex = e % E, ey = (e / E) % E, ez = e / (E * E);
            int gx = (tx0 - m + 1 + ex) & msk, gy = (ty0 - m + 1 + ey) & msk,
                gz = (tz0 - m + 1 + ez) & msk;
            S[e] = __ldg(&gl[((int64_t)gz * n + gy) * n + gx]);
        }
        __syncthreads();
        ChunkCursor cur = make_cursor(s_items, team, nit);
        if (cur.valid()) st.issue(0, wts, cur);
        int pcur = (cur.valid() && lane < cur.cnt) ? perm[cur.start + lane] : 0;
        uint32_t ah[4][4], al[4][4];  // the item's stencil, A = G[(z, y), x]
        int bsel = 0;
        while (cur.valid()) {
            if (cur.c0 == 0) {
                int lx0, ly0, lz0;
                item_local(cur.local, lx0, ly0, lz0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float *r0 = S + ((lz0 + 2 * i) * E + (ly0 + g)) * E + lx0;
                    const float *r1 = S + ((lz0 + 2 * i + 1) * E + (ly0 + g)) * E + lx0;
                    tf32_split(r0[t], ah[i][0], al[i][0]);
                    tf32_split(r1[t], ah[i][1], al[i][1]);
                    tf32_split(r0[t + 4], ah[i][2], al[i][2]);
                    tf32_split(r1[t + 4], ah[i][3], al[i][3]);
                }
            }
            const ChunkCursor nxt = next_chunk<NW>(cur, s_items, nit, s_ctl, s_slot, team, tid);
            int pnxt = 0;
            if (nxt.valid()) {
                st.issue(bsel ^ 1, wts, nxt);
                if (lane < nxt.cnt - nxt.c0) pnxt = perm[nxt.start + nxt.c0 + lane];
            }
            if (!st.wait(bsel, err)) {
                st.drain(err);
                s_ctl[2] = 1;
                break;
            }
            const float *sw = st.buf(bsel);
            const int cn = min(kChunk, cur.cnt - cur.c0);
            for (int g0 = 0; g0 < cn; g0 += 8) {
                // B: k = x (t, t + 4), n = point g0 + g
                const int pb = g0 + g;
                const float *wb = sw + (pb < cn ? pb : g0) * PWP;
                uint32_t bh0, bl0, bh1, bl1;
                tf32_split(pb < cn ? wb[t] : 0.f, bh0, bl0);
                tf32_split(pb < cn ? wb[t + 4] : 0.f, bh1, bl1);
                float c[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
                    mma_3xtf32(c[i], ah[i], al[i], bh0, bh1, bl0, bl1);
                }
                // this thread: y = g, z = 0..7, points q0 = g0 + 2t, q1 = q0 + 1
                const int q0 = g0 + 2 * t, q1 = q0 + 1;
                const float *w0 = sw + (q0 < cn ? q0 : g0) * PWP;
                const float *w1 = sw + (q1 < cn ? q1 : g0) * PWP;
                const float4 z0a = *reinterpret_cast<const float4 *>(w0 + 2 * W2);
                const float4 z0b = *reinterpret_cast<const float4 *>(w0 + 2 * W2 + 4);
                const float4 z1a = *reinterpret_cast<const float4 *>(w1 + 2 * W2);
                const float4 z1b = *reinterpret_cast<const float4 *>(w1 + 2 * W2 + 4);
                const float wz0[8] = {z0a.x, z0a.y, z0a.z, z0a.w, z0b.x, z0b.y, z0b.z, z0b.w};
                const float wz1[8] = {z1a.x, z1a.y, z1a.z, z1a.w, z1b.x, z1b.y, z1b.z, z1b.w};
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    s0 = fmaf(wz0[2 * i], c[i][0], s0);
                    s0 = fmaf(wz0[2 * i + 1], c[i][2], s0);
                    s1 = fmaf(wz1[2 * i], c[i][1], s1);
                    s1 = fmaf(wz1[2 * i + 1], c[i][3], s1);
                }
                s0 *= w0[W2 + g];
                s1 *= w1[W2 + g];
                // sum over y = g: lanes 4 g + t with the same t
#pragma unroll
                for (int o = 4; o <= 16; o <<= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                }
                const int pi0 = __shfl_sync(0xffffffffu, pcur, q0 & 31);
                const int pi1 = __shfl_sync(0xffffffffu, pcur, q1 & 31);
                if (g == 0) {
                    if (q0 < cn) Y[(int64_t)l * N + pi0] = (double)s0;
                    if (q1 < cn) Y[(int64_t)l * N + pi1] = (double)s1;
                }
            }
            __syncwarp();  // every read of buffer bsel is done before it is refilled
            cur = nxt;
            pcur = pnxt;
            bsel ^= 1;
        }
    }
}

// xs[s] = x[perm[s]] for every sorted position s (input in sorted order).
template <typename T>
__global__ void k_gather(const double *__restrict__ x, const int *__restrict__ perm, int64_t LN,
                         T *__restrict__ xs, const int *__restrict__ done) {
    if (done && *done) return;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < LN;
         s += (int64_t)gridDim.x * blockDim.x)
        xs[s] = (T)x[perm[s]];
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
k_conv(typename Num<T>::G *__restrict__ grid, int axis, const T *__restrict__ tab,
       const typename Vec2<T>::type *__restrict__ tw, const int *__restrict__ done) {
    using G = typename Num<T>::G;
    using C = typename Vec2<T>::type;
    constexpr int n = 32 * R, LPC = 16, PITCH = n + 1;
    __shared__ T S[LPC * PITCH];
    if (done && *done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    G *g = grid + (int64_t)blockIdx.y * n * n * n;
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
            S[j * PITCH + e] = T(g[goff(j, e)]);
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            S[j * PITCH + e] = T(g[goff(j, e)]);
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
            g[goff(j, e)] = (G)S[j * PITCH + e];
        }
    } else {
        for (int q = tid; q < LPC * n; q += 256) {
            int j = q % LPC, e = q / LPC;
            g[goff(j, e)] = (G)S[j * PITCH + e];
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
           const double *__restrict__ d, double alpha_val, const double *__restrict__ alpha_dev,
           int op, double *__restrict__ y,
           double *__restrict__ partials, T *__restrict__ grid, int64_t grid_elems,
           int *__restrict__ unit_ctr, const int *__restrict__ done) {
    __shared__ double sh[33];
    if (done && *done) return;
    const double alpha = alpha_dev ? *alpha_dev : alpha_val;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unit_ctr[0] = 0;  // the spread and interpolation kernels have finished
        unit_ctr[1] = 0;
    }
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
template <typename T> constexpr int spread_class() {
    return sizeof(T) == 4 ? NLH_K_SPREAD32 : (Num<T>::kParts == 2 ? NLH_K_SPREADDF : NLH_K_SPREAD64);
}


template <typename T, int W2, int NW, int TPB>
static void launch_spread_interp_shape(Plan &P, bool spread, const typename Num<T>::R *wts,
                                 typename Num<T>::G *grid, const T *xs, const int *done,
                                 cudaStream_t s) {
    constexpr int NTH = 32 * NW * TPB;
    // the FP32 2m = 8 default shape with registers capped for 5 CTAs per SM
    // (no spills; 1% faster matvecs than the uncapped 4 CTAs)
    constexpr int MINB =
        (std::is_same<T, float>::value && W2 == 8 && NW == 1 && TPB == 4) ? 5 : 1;
    constexpr size_t smem = UnitLayout<T, W2, TPB>::bytes;
    if (P.units_cap == 0) return;
    static int blocks_spread = 0, blocks_interp = 0;  // per template instance
    if (blocks_spread == 0) {
        NLH_CUDA(cudaFuncSetAttribute(k_spread<T, W2, NW, TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NLH_CUDA(cudaFuncSetAttribute(k_interp<T, W2, NW, TPB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0, a = 0, b = 0;
        NLH_CUDA(cudaGetDevice(&dev));
        NLH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spread<T, W2, NW, TPB, MINB>,
                                                               NTH, smem));
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_interp<T, W2, NW, TPB>, NTH,
                                                               smem));
        blocks_interp = sms * std::max(1, b);
        blocks_spread = sms * std::max(1, a);
    }
    ProfRange pr(spread ? spread_class<T>() : interp_class<T>(), s);
    // grid bound: the unit count once known on the host, else its upper bound
    const int64_t nu = P.n_units >= 0 ? P.n_units : P.units_cap;
    if (nu == 0) return;
    if (spread) {
        const unsigned g = (unsigned)std::min<int64_t>(blocks_spread, nu);
        k_spread<T, W2, NW, TPB, MINB><<<g, NTH, smem, s>>>(P.units, P.d_units, P.unit_ctr, P.items,
                                                            wts, xs, grid, P.n, P.m, done, P.err);
    } else {
        const unsigned g = (unsigned)std::min<int64_t>(blocks_interp, nu);
        k_interp<T, W2, NW, TPB><<<g, NTH, smem, s>>>(P.units, P.d_units, P.unit_ctr + 1, P.items,
                                                      P.perm, wts, grid, P.Y, P.n, P.m, P.N, done,
                                                      P.err);
    }
    NLH_CHECK_LAUNCH();
}

// The tensor-core FP32 kernels (2m = 8, one-warp teams, 4 teams per CTA,
// registers capped for MINB resident CTAs per SM).
template <int MINB>
static void launch_spread_interp_tc(Plan &P, bool spread, const float *wts, float *grid,
                                    const float *xs, const int *done, cudaStream_t s) {
    constexpr int TPB = 4, NTH = 32 * TPB;
    constexpr size_t smem = UnitLayout<float, 8, TPB>::bytes;
    if (P.units_cap == 0) return;
    static int blocks_spread = 0, blocks_interp = 0;
    if (blocks_spread == 0) {
        NLH_CUDA(cudaFuncSetAttribute(k_spread_tc<TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NLH_CUDA(cudaFuncSetAttribute(k_interp_tc<TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int dev = 0, sms = 0, a = 0, b = 0;
        NLH_CUDA(cudaGetDevice(&dev));
        NLH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spread_tc<TPB, MINB>, NTH,
                                                               smem));
        NLH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_interp_tc<TPB, MINB>, NTH,
                                                               smem));
        blocks_interp = sms * std::max(1, b);
        blocks_spread = sms * std::max(1, a);
    }
    ProfRange pr(spread ? NLH_K_SPREAD32 : NLH_K_INTERP32, s);
    const int64_t nu = P.n_units >= 0 ? P.n_units : P.units_cap;
    if (nu == 0) return;
    if (spread) {
        const unsigned g = (unsigned)std::min<int64_t>(blocks_spread, nu);
        k_spread_tc<TPB, MINB><<<g, NTH, smem, s>>>(P.units, P.d_units, P.unit_ctr, P.items, wts,
                                                    xs, grid, P.n, P.m, done, P.err);
    } else {
        const unsigned g = (unsigned)std::min<int64_t>(blocks_interp, nu);
        k_interp_tc<TPB, MINB><<<g, NTH, smem, s>>>(P.units, P.d_units, P.unit_ctr + 1, P.items,
                                                    P.perm, wts, grid, P.Y, P.n, P.m, P.N, done,
                                                    P.err);
    }
    NLH_CHECK_LAUNCH();
}

template <typename T> constexpr int arith_index() {
    return sizeof(T) == 8 && !std::is_same<T, df32>::value ? NLH_FP64
           : std::is_same<T, df32>::value                   ? NLH_DF32
                                                            : NLH_FP32;
}

// Team shape (warps per team NW, teams per CTA TPB) of the spread and
// interpolation kernels: fewer accumulator lines per thread (larger teams)
// against more independent teams per SM.  Shape 0 is the default; shapes 1
// and 2 are compiled for the stencil widths of the workloads (2m = 8, 12);
// shape 3 is the tensor-core FP32 path for 2m = 8.  The autotuner picks one
// per arithmetic (plan.team[]); other combinations fall back to shape 0.
template <typename T, int W2>
static void launch_spread_interp(Plan &P, bool spread, const typename Num<T>::R *wts,
                                 typename Num<T>::G *grid, const T *xs, const int *done,
                                 cudaStream_t s) {
    const int shape = P.team[arith_index<T>()];
    // interpolation: points on lanes unless the plan asks for the team kernel
    // (or the tensor-core FP32 shape, which has its own).  Compiled for the
    // stencil widths of the workloads (2m = 8, 12): its fully unrolled
    // stencil makes every further width a long compile; other widths run
    // the team kernel.
    if constexpr (W2 == 8 || W2 == 12) {
        if (!spread && P.interp_kind == NLH_INTERP_POINTS && shape != 3)
            return launch_interp_pl<T, W2>(P, wts, grid, done, s);
    }
    if constexpr (W2 == 8 && std::is_same<T, float>::value) {
        if (shape == 3) return launch_spread_interp_tc<5>(P, spread, wts, grid, xs, done, s);
    }
    if constexpr (W2 == 8) {
        if (shape == 1) return launch_spread_interp_shape<T, W2, 2, 2>(P, spread, wts, grid, xs, done, s);
        if (shape == 2) return launch_spread_interp_shape<T, W2, 2, 4>(P, spread, wts, grid, xs, done, s);
    } else if constexpr (W2 == 12) {
        if (shape == 1) return launch_spread_interp_shape<T, W2, 4, 1>(P, spread, wts, grid, xs, done, s);
        if (shape == 2) return launch_spread_interp_shape<T, W2, 2, 1>(P, spread, wts, grid, xs, done, s);
    }
    constexpr int NW = W2 <= 8 ? 1 : 2, TPB = W2 <= 8 ? 4 : 2;
    launch_spread_interp_shape<T, W2, NW, TPB>(P, spread, wts, grid, xs, done, s);
}

template <typename T>
static void spread_interp(Plan &P, bool spread, const typename Num<T>::R *wts,
                          typename Num<T>::G *grid, const T *v, const int *done, cudaStream_t s) {
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
static void convolve(Plan &P, typename Num<T>::G *grid, const T *tab,
                     const typename Vec2<T>::type *tw, const int *done, cudaStream_t s) {
    const int n = P.n;
    dim3 gdim((unsigned)(n * n / 16), (unsigned)P.L);
    ProfRange pr(sizeof(T) == 4 ? NLH_K_CONV32 : NLH_K_CONV64, s);
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

// One matvec in arithmetic T: gather the input into sorted order, spread,
// convolve the grids, interpolate, and the epilogue (which also clears the
// grids and the unit counters for the next matvec).
template <typename T>
static void matvec_t(Plan &P, int op, double alpha, const double *alpha_dev, const double *x,
                     double *y, double *partials, const int *done,
                     const typename Num<T>::R *wts, typename Num<T>::G *grid, const T *tab,
                     const typename Vec2<T>::type *tw, const double *d, cudaStream_t s) {
    using G = typename Num<T>::G;
    T *xs = reinterpret_cast<T *>(P.xs);
    {
        ProfRange pr(NLH_K_EPILOGUE, s);
        k_gather<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, P.perm, (int64_t)P.L * P.N, xs, done);
        NLH_CHECK_LAUNCH();
    }
    spread_interp<T>(P, true, wts, grid, xs, done, s);
    convolve<T>(P, grid, tab, tw, done, s);
    spread_interp<T>(P, false, wts, grid, nullptr, done, s);
    const int64_t ge = (int64_t)P.L * P.n * P.n * P.n;
    ProfRange pr(NLH_K_EPILOGUE, s);
    k_epilogue<G><<<kRedBlocks, kRedThreads, 0, s>>>(P.Y, P.L, P.N, x, d, alpha, alpha_dev, op, y,
                                                     partials, grid, ge, P.unit_ctr, done);
    NLH_CHECK_LAUNCH();
}

void matvec(Plan &P, int op, int prec, double alpha, const double *x, double *y,
            double *partials, const int *done, cudaStream_t s, const double *alpha_dev) {
    if (prec == NLH_FP64) {
        NLH_REQUIRE(P.precision & 1, "matvec: FP64 path not built in this plan");
        matvec_t<double>(P, op, alpha, alpha_dev, x, y, partials, done, P.wts64, P.grid64,
                         P.tab64, P.tw64, P.d64, s);
    } else if (prec == NLH_FP32) {
        NLH_REQUIRE(P.precision & 2, "matvec: FP32 path not built in this plan");
        matvec_t<float>(P, op, alpha, alpha_dev, x, y, partials, done, P.wts32, P.grid32,
                        P.tab32, P.tw32, P.d32, s);
    } else {
        NLH_REQUIRE(P.precision & 4, "matvec: double-float path not built in this plan");
        matvec_t<df32>(P, op, alpha, alpha_dev, x, y, partials, done, P.wtsdf, P.grid64,
                       reinterpret_cast<const df32 *>(P.tabdf),
                       reinterpret_cast<const cdf *>(P.twdf), P.ddf, s);
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
        NLH_REQUIRE(precision == NLH_FP64 || precision == NLH_FP32 || precision == NLH_DF32,
                    "nlh_matvec: precision=%d", precision);
        plan->stream = (cudaStream_t)stream;
        nlh::matvec(*plan, op, precision, alpha, x, y, nullptr, nullptr, (cudaStream_t)stream);
        return NLH_OK;
    } catch (nlh::Failure &f) {
        return f.st;
    }
}
