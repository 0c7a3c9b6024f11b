// df32.cuh -- FP64-accurate arithmetic on the FP32 pipes ("double-float").
//
// A value is an unevaluated sum hi + lo of two floats.  Products use the
// exact-product property of a fused multiply-add (the error of hi*hi is
// fma(a, b, -a*b), Dekker 1971; with an FMA this is the standard TwoProduct),
// sums use Knuth's TwoSum (The Art of Computer Programming, vol. 2, 4.2.2),
// and the low parts are accumulated in plain FP32, which keeps about 46-48
// significant bits.  The explicit _rn intrinsics stop the compiler from
// contracting the error terms.  Results are left unnormalised (|lo| may be a
// few ulps of hi); conversion back to double is hi + lo.
//
// GB300 runs FP32 FMAs 59x faster than FP64 FMAs (measured 70 vs 1.19
// TFLOP/s), so an FP64-accurate NFFT evaluated this way is several times
// faster than native FP64, at the cost of ~2^-46 relative rounding instead of
// 2^-53.
#pragma once
#include <cstdint>

namespace nlh {

struct df32 {
    float hi, lo;
    df32() = default;
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit df32(double x)
        : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit df32(int x) : hi((float)x), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// TwoProduct with the cross terms of the low parts; unnormalised result.
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df32(p, e);
}

// TwoSum of the high parts; low parts added in FP32.
__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bp = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
    return df32(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }

__device__ __forceinline__ df32 &operator+=(df32 &a, df32 b) {
    a = a + b;
    return a;
}
__device__ __forceinline__ df32 &operator*=(df32 &a, df32 b) {
    a = a * b;
    return a;
}

// Complex double-float (FFT data and twiddles).
struct cdf {
    df32 x, y;
};

__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) { return a * b + c; }

__device__ __forceinline__ bool operator!=(df32 a, df32 b) { return a.hi != b.hi || a.lo != b.lo; }

__device__ __forceinline__ df32 __shfl_sync(unsigned mask, df32 v, int src) {
    return df32(::__shfl_sync(mask, v.hi, src), ::__shfl_sync(mask, v.lo, src));
}
__device__ __forceinline__ df32 __shfl_xor_sync(unsigned mask, df32 v, int o) {
    return df32(::__shfl_xor_sync(mask, v.hi, o), ::__shfl_xor_sync(mask, v.lo, o));
}

// Compensated atomic accumulation: the float atomic on the high part returns
// the old value, from which the rounding error of that very addition is
// recovered by TwoSum and added, with the low part, into the low word.
// (FP32 atomics round to nearest even, as __fadd_rn does; subnormals flush
// to zero, which only touches values below 1.2e-38.)
__device__ __forceinline__ void atomicAdd(df32 *addr, df32 v) {
    float old = ::atomicAdd(&addr->hi, v.hi);
    float s = __fadd_rn(old, v.hi);
    float bp = __fsub_rn(s, old);
    float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bp)), __fsub_rn(v.hi, bp));
    ::atomicAdd(&addr->lo, __fadd_rn(err, v.lo));
}

// The df32 overloads above would hide the global functions of the same
// names inside this namespace; bring those back into the overload sets.
using ::atomicAdd;
using ::fma;
using ::__shfl_sync;
using ::__shfl_xor_sync;

// ---- packed pairs: one 64-bit register holds two floats (two grid cells)
__device__ __forceinline__ unsigned long long pk_dup(float x) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void pk_split(unsigned long long v, float &lo_half, float &hi_half) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo_half), "=f"(hi_half) : "l"(v));
}
__device__ __forceinline__ unsigned long long pk_make(float lo_half, float hi_half) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo_half), "f"(hi_half));
    return r;
}
__device__ __forceinline__ unsigned long long pk_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long pk_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long pk_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long pk_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// (h, l) += (a.hi, a.lo) * (wh, wl) for two cells at once.  nah, nal are
// the negated (duplicated) parts of a; the product's error term is formed
// negated, e = p - a*w = fma(-a, w, p), so that it only needs fused
// multiply-adds.  (The other form, fma(a, w, 0 - p) on the packed
// instructions, measured on sm_103a with CUDA 13.0 as if the product's
// rounding error were zero; the negated-operand form is exact.)
__device__ __forceinline__ void pk_df_axpy(unsigned long long &h, unsigned long long &l,
                                           unsigned long long ah, unsigned long long nah,
                                           unsigned long long nal, unsigned long long wh,
                                           unsigned long long wl) {
    unsigned long long p = pk_mul(ah, wh);
    unsigned long long e = pk_fma(nah, wh, p);
    e = pk_fma(nah, wl, e);
    e = pk_fma(nal, wh, e);
    unsigned long long s = pk_add(h, p);
    unsigned long long bp = pk_sub(s, h);
    unsigned long long t = pk_add(pk_sub(h, pk_sub(s, bp)), pk_sub(p, bp));
    l = pk_add(l, pk_sub(t, e));
    h = s;
}

}  // namespace nlh
