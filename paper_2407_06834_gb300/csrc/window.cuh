// window.cuh -- Kaiser-Bessel window weights evaluated in registers.
//
// The window (Kaiser 1974; its use for gridding: Jackson et al. 1991) is
//   phi(x) = I0(beta sqrt(1 - (n x / m)^2)) / I0(beta),  |n x| <= m,
// with beta = pi m (2 - M / n) (Sec. 3: the NFFT's window function; the
// parameters follow the oversampling of the plan).  A point at grid
// coordinate u = c + f (c the cell, 0 <= f < 1) touches the 2m grid points
// c - m + 1 + j, j = 0 .. 2m - 1, with weight P_j(f) = phi((j - m + 1 - f) / m).
// In y = 2 f - 1 the weights come in mirrored pairs: P_{2m-1-j}(y) = P_j(-y),
// so with P_j(y) = E_j(y^2) + y O_j(y^2) one evaluation of the even part E_j
// and the odd part O_j gives both weights of a pair:
//   w_j = E_j + y O_j,   w_{2m-1-j} = E_j - y O_j.
// E_j and O_j are fitted once per (m, beta) on the host (Chebyshev
// interpolation of P_j, converted to monomials; plan.cu).  The FP32 set
// reaches the kernels as a small by-value kernel parameter read at
// compile-time offsets only, so every coefficient is a constant operand of
// the multiply-adds; the FP64 and double-float sets are staged from a table
// in the plan's device memory into shared memory.  Per point and dim this
// is m pairs of short Horner chains instead of a stored weight record.
#pragma once
#include <cstdint>

#include "df32.cuh"

namespace nlh {

constexpr int kWinHalfMax = 8;  // m <= 8
constexpr int kWinK32 = 5;      // coefficients of E_j and of O_j, FP32 (degree-9 fit)
constexpr int kWinK64 = 8;      // coefficients of E_j and of O_j, FP64 / double-float (degree 15)
// Double-float chains start in FP32 for the coefficients k >= kWinDfSplit
// (in powers of y^2): their sum is below 1e-7 for every (m, beta) the plans
// use, so the FP32 rounding of that part stays below ~1e-14.
constexpr int kWinDfSplit = 5;

template <typename T> struct WinPoly;
template <> struct WinPoly<float> {
    float c[kWinHalfMax][2][kWinK32];  // [j][0: even, 1: odd][power of y^2]
};
template <> struct WinPoly<double> {
    double c[kWinHalfMax][2][kWinK64];
};
template <> struct WinPoly<df32> {
    float hi[kWinHalfMax][2][kWinK64], lo[kWinHalfMax][2][kWinK64];
};

// The 2m weights of one dim at y = 2 f - 1, FP32.
template <int W2>
__device__ __forceinline__ void win_weights(const WinPoly<float> &c, float y, float (&w)[W2]) {
    const float u = y * y;
#pragma unroll
    for (int j = 0; j < W2 / 2; ++j) {
        float e = c.c[j][0][kWinK32 - 1], o = c.c[j][1][kWinK32 - 1];
#pragma unroll
        for (int k = kWinK32 - 2; k >= 0; --k) {
            e = fmaf(e, u, c.c[j][0][k]);
            o = fmaf(o, u, c.c[j][1][k]);
        }
        w[j] = fmaf(y, o, e);
        w[W2 - 1 - j] = fmaf(-y, o, e);
    }
}

// FP64, coefficients from the shared-memory copy of the plan's staged
// table: sc[j][k] = {E_k, O_k} (the same register pressure as for
// double-float).
template <int W2>
__device__ __forceinline__ void win_weights(const double2 *sc, double y, double (&w)[W2]) {
    const double u = y * y;
#pragma unroll
    for (int j = 0; j < W2 / 2; ++j) {
        const double2 t = sc[j * kWinK64 + kWinK64 - 1];
        double e = t.x, o = t.y;
#pragma unroll
        for (int k = kWinK64 - 2; k >= 0; --k) {
            const double2 q = sc[j * kWinK64 + k];
            e = fma(e, u, q.x);
            o = fma(o, u, q.y);
        }
        w[j] = fma(y, o, e);
        w[W2 - 1 - j] = fma(-y, o, e);
    }
}

// Double-float: the leading coefficients in FP32, the rest as Horner steps
// w = w u + c with TwoProduct / TwoSum (df32.cuh).  The even and odd chains
// of a pair run side by side in packed f32x2 registers (both multiply by the
// same u), one instruction per step for both.  TwoSum reads each
// coefficient several times, and a compiler that keeps all of them in
// registers across a kernel's loops runs out of registers, so the
// coefficients come from a shared-memory copy of the plan's staged table,
// one broadcast 16-byte load per step: sc[j][k] = {E hi, O hi, E lo, O lo}.
// Bytes of one staged table: kWinK64 16-byte entries per j, {E_k, O_k} as
// doubles (FP64) or {E hi, O hi, E lo, O lo} as floats (double-float).
constexpr int kWinStageBytes = 16 * kWinHalfMax * kWinK64;

// Copies a staged table (global memory, kWinStageBytes) into shared memory.
__device__ __forceinline__ void win_stage(const float4 *__restrict__ src, float4 *sc) {
    for (int e = threadIdx.x; e < kWinStageBytes / 16; e += blockDim.x) sc[e] = __ldg(src + e);
}

template <int W2>
__device__ __forceinline__ void win_weights(const float4 *sc, df32 y, df32 (&w)[W2]) {
    const df32 u = y * y;
    // u and its negation, duplicated into both halves; the product errors are
    // formed negated, p - h u, with the negated u as an operand (as in
    // pk_df_axpy), so that they need fused multiply-adds only
    const unsigned long long uh = pk_dup(u.hi), nuh = pk_dup(-u.hi), nul = pk_dup(-u.lo);
    const ulonglong2 *sq = reinterpret_cast<const ulonglong2 *>(sc);
#pragma unroll
    for (int j = 0; j < W2 / 2; ++j) {
        // h = (E hi, O hi), l = (E lo, O lo)
        unsigned long long h = sq[j * kWinK64 + kWinK64 - 1].x, l = 0ull;
#pragma unroll
        for (int k = kWinK64 - 2; k >= kWinDfSplit; --k) h = pk_fma(h, uh, sq[j * kWinK64 + k].x);
#pragma unroll
        for (int k = kWinDfSplit - 1; k >= 0; --k) {
            const ulonglong2 q = sq[j * kWinK64 + k];
            // (h, l) * (u hi, u lo): product p and its negated error ne with the
            // cross terms
            const unsigned long long p = pk_mul(h, uh);
            unsigned long long ne = pk_fma(h, nuh, p);
            ne = pk_fma(h, nul, ne);
            ne = pk_fma(l, nuh, ne);
            // + (c hi, c lo): TwoSum of the high parts, low parts in FP32
            const unsigned long long s2 = pk_add(p, q.x);
            const unsigned long long bp = pk_sub(s2, p);
            const unsigned long long t = pk_add(pk_sub(p, pk_sub(s2, bp)), pk_sub(q.x, bp));
            l = pk_add(t, pk_sub(q.y, ne));
            h = s2;
        }
        float eh, oh, el, ol;
        pk_split(h, eh, oh);
        pk_split(l, el, ol);
        const df32 yo = y * df32(oh, ol);
        const df32 e = df32(eh, el);
        w[j] = e + yo;
        w[W2 - 1 - j] = e - yo;
    }
}

// One signature for the kernels: the FP32 form reads its by-value parameter
// set, the FP64 and double-float forms the staged shared-memory table.
struct NoPoly {};
template <typename T> struct PolyArg { using type = NoPoly; };
template <> struct PolyArg<float> { using type = WinPoly<float>; };

template <int W2>
__device__ __forceinline__ void win_weights(const WinPoly<float> &c, const float4 *, float y,
                                            float (&w)[W2]) {
    win_weights<W2>(c, y, w);
}
template <int W2>
__device__ __forceinline__ void win_weights(const NoPoly &, const float4 *sc, double y,
                                            double (&w)[W2]) {
    win_weights<W2>(reinterpret_cast<const double2 *>(sc), y, w);
}
template <int W2>
__device__ __forceinline__ void win_weights(const NoPoly &, const float4 *sc, df32 y,
                                            df32 (&w)[W2]) {
    win_weights<W2>(sc, y, w);
}

}  // namespace nlh
