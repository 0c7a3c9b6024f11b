// net.cu -- the learned warm start and diagonal correction (no counterpart
// in the paper; the network definition is in include/nlh_net.h).
//
// Layouts.  Activations NHWC bfloat16 (channels contiguous); the input
// planes are padded to 32 channels.  Gradients of activations NHWC float.
// Canonical FP32 parameters per 3x3 layer W[cout][3][3][cin], b[cout]; head
// W[2][base], b[2].  GEMM copies of the 3x3 weights in bfloat16: forward
// Wf[cout][9][cin32] and input-gradient Wd[cin32][9][cout] (cin32 = cin
// rounded up to 32; the padding is zero).
//
// Kernels.
//   k_conv3x3<BN>    implicit GEMM on the tensor cores (mma.sync m16n8k16,
//                    bf16 x bf16 -> f32): M = pixels (128 per CTA), N =
//                    output channels (BN per CTA), K = 9 taps x input
//                    channels in 32-channel chunks.  The A rows are the
//                    shifted input pixels (zero outside the image; the
//                    source is either one tensor, or the concatenation of an
//                    upsampled coarse tensor and a skip tensor, resolved per
//                    chunk), staged with cp.async in a 3-stage pipeline into
//                    XOR-swizzled shared memory and read with ldmatrix.
//                    Forward: +bias, ReLU, bf16 out.  Input gradient: the
//                    same GEMM with the taps mirrored (input = out - offset)
//                    and Wd, f32 out, optionally split into two tensors at a
//                    channel boundary (the two parts of a concatenation).
//   k_conv3x3_tc<BN> the same forward / input-gradient GEMM on tcgen05 (the
//                    default engine): M runs over the zero-padded image's
//                    pixels, so one staged band of 130 pixels serves the
//                    three horizontal taps of a row offset; the accumulator
//                    is in tensor memory, read back with tcgen05.ld.
//   k_conv3x3_wgrad_tc<MT> the weight gradient on tcgen05 (the default
//                    engine): M = output channels, N = 32 input channels,
//                    K = padded pixels, both operands MN-major, the input
//                    band shared by the three horizontal taps as in the
//                    forward kernel; split K with f32 atomics.
//   k_conv3x3_wgrad  weight gradient dW[co][tap][ci] = sum_p dZ[p][co]
//                    X[p + off(tap)][ci]: M = cout, N = 32 input channels of
//                    one tap, K = pixels split across CTAs, both operands
//                    read with ldmatrix.trans; f32 atomics into the
//                    canonical gradient.
//   k_grad_merge     the gradient reaching a ReLU output (same-resolution,
//                    average-pool backward from the coarser level, upsample
//                    backward from the finer level), masked by y > 0, to
//                    bf16, with the bias gradient reduced on the fly.
//   k_input_planes, k_avgpool2, k_stats_partial / k_stats_final, k_head_fwd, k_loss_grad,
//   k_head_bwd, k_adam, k_pack_weights, k_sub.
#include "common.cuh"
#include "async_copy.cuh"
#include "../../include/nlh_net.h"
#include "../../include/nlh_selftest.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

namespace nlh {
namespace netk {

using bf16 = __nv_bfloat16;

constexpr int kMaxBatch = 64;
constexpr int kBM = 128;      // pixels per forward / input-gradient CTA
constexpr int kBK = 32;       // channels per K chunk
constexpr int kStages = 3;    // cp.async pipeline depth
constexpr int kConvThreads = 128;
constexpr int kElemThreads = 256;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte global -> shared copy; zero-filled (no global read) when !valid.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                          uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// D += A (16x16, row) * B (16x8, col), bf16 inputs, f32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// XOR swizzle of the 16-byte chunk c in a shared-memory row of CPR chunks:
// the 8 rows an ldmatrix phase reads at one logical chunk land in 8
// distinct 16-byte bank groups.
template <int CPR> __device__ __forceinline__ int swz(int row, int c) {
    static_assert(CPR == 4 || CPR % 8 == 0, "rows of 4 or 8k chunks");
    if constexpr (CPR == 4)
        return c ^ ((row >> 1) & 3);
    else
        return c ^ (row & 7);
}

// ------------------------------------------------------------ input sources
// The input of a 3x3 convolution: channels [0, c1) from x1 (at half
// resolution when up1, read at (y >> 1, x >> 1): nearest upsampling),
// channels [c1, c1 + c2) from x2 (full resolution).  c1, c2 multiples of 32.
struct Src {
    const bf16 *x1;
    int c1, up1;
    const bf16 *x2;
    int c2;
};

// Address of channels c .. c+7 of input pixel (b, y, x), or nullptr outside
// the H x W image (zero padding).
__device__ __forceinline__ const bf16 *src_ptr(const Src &s, int b, int y, int x, int H, int W,
                                               int c) {
    if (y < 0 || y >= H || x < 0 || x >= W) return nullptr;
    if (c < s.c1) {
        const int Hs = H >> s.up1, Ws = W >> s.up1;
        return s.x1 + (((int64_t)b * Hs + (y >> s.up1)) * Ws + (x >> s.up1)) * s.c1 + c;
    }
    return s.x2 + (((int64_t)b * H + y) * W + x) * s.c2 + (c - s.c1);
}

// ------------------------------------------------- forward / input gradient
struct ConvArgs {
    Src src;
    const bf16 *w;      // [n][9][cin], cin = c1 + c2
    const bf16 *wt;     // the same weights as [9][cin / 32][4][n][8] (tcgen05 engine)
    const float *bias;  // [n] or nullptr
    int relu;
    int sign;           // +1: input pixel = output + offset; -1: output - offset
    int B, H, W;
    int n;              // output channels
    bf16 *ybf;          // bf16 output [P][n], or nullptr for float output
    float *y1;          // float output channels [0, n1) -> y1 [P][n1]
    int n1;
    float *y2;          // channels [n1, n) -> y2 [P][n - n1]
};

template <int BN>
__global__ void __launch_bounds__(kConvThreads) k_conv3x3(ConvArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int A_BYTES = kBM * kBK * 2;
    constexpr int B_BYTES = BN * kBK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr int WN = BN / 2;   // columns per warp (2 x 2 warps)
    constexpr int NB = WN / 8;   // n8 blocks per warp
    static_assert(NB % 2 == 0, "B fragments are loaded in pairs");

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HW = a.H * a.W;
    const int64_t P = (int64_t)a.B * HW;
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const int cin = a.src.c1 + a.src.c2;
    const int kcb = cin / kBK;
    const int nk = 9 * kcb;

    // the A row this thread stages: pixel m0 + tid
    const int64_t m = m0 + tid;
    const bool mvalid = m < P;
    int pb = 0, py = 0, px = 0;
    if (mvalid) {
        pb = (int)(m / HW);
        const int rem = (int)(m - (int64_t)pb * HW);
        py = rem / a.W;
        px = rem - py * a.W;
    }

    auto load = [&](int stage, int kc) {
        const int tap = kc / kcb, cb = kc - tap * kcb;
        const int dy = (tap / 3 - 1) * a.sign, dx = (tap % 3 - 1) * a.sign;
        const int c0 = cb * kBK;
        const uint32_t sa = smem_u32(smem + stage * STAGE);
        const uint32_t sb = sa + A_BYTES;
        const bf16 *p = mvalid ? src_ptr(a.src, pb, py + dy, px + dx, a.H, a.W, c0) : nullptr;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            cp_async16(sa + (tid * 4 + swz<4>(tid, q)) * 16, p ? p + 8 * q : a.w, p != nullptr);
#pragma unroll
        for (int i = 0; i < BN * 4 / kConvThreads; ++i) {
            const int idx = tid + i * kConvThreads;
            const int r = idx >> 2, q = idx & 3;
            const bf16 *wp = a.w + ((int64_t)(n0 + r) * 9 + tap) * cin + c0 + 8 * q;
            cp_async16(sb + (r * 4 + swz<4>(r, q)) * 16, wp, true);
        }
    };

    float acc[4][NB][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NB; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const int wm = warp & 1, wn = warp >> 1;

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load(s, s);
        cp_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        cp_wait<kStages - 2>();
        __syncthreads();
        {
            const int nx = kc + kStages - 1;
            if (nx < nk) load(nx % kStages, nx);
            cp_commit();
        }
        const uint32_t sa = smem_u32(smem + (kc % kStages) * STAGE);
        const uint32_t sb = sa + A_BYTES;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t af[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = wm * 64 + i * 16 + (lane & 15);
                const int ch = ks * 2 + (lane >> 4);
                ldsm_x4(sa + (row * 4 + swz<4>(row, ch)) * 16, af[i][0], af[i][1], af[i][2],
                        af[i][3]);
            }
#pragma unroll
            for (int j = 0; j < NB / 2; ++j) {
                const int row = wn * WN + j * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int ch = ks * 2 + ((lane >> 3) & 1);
                uint32_t b0, b1, b2, b3;
                ldsm_x4(sb + (row * 4 + swz<4>(row, ch)) * 16, b0, b1, b2, b3);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    mma_bf16(acc[i][2 * j], af[i], b0, b1);
                    mma_bf16(acc[i][2 * j + 1], af[i], b2, b3);
                }
            }
        }
    }
    cp_wait<0>();

    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t mm = m0 + wm * 64 + i * 16 + g + h * 8;
            if (mm >= P) continue;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const int n = n0 + wn * WN + j * 8 + 2 * t;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[n];
                    v1 += a.bias[n + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (a.ybf)
                    *reinterpret_cast<__nv_bfloat162 *>(a.ybf + mm * a.n + n) =
                        __floats2bfloat162_rn(v0, v1);
                else if (n < a.n1)
                    *reinterpret_cast<float2 *>(a.y1 + mm * a.n1 + n) = make_float2(v0, v1);
                else
                    *reinterpret_cast<float2 *>(a.y2 + mm * (a.n - a.n1) + (n - a.n1)) =
                        make_float2(v0, v1);
            }
        }
    }
}

// ------------------------------------- forward / input gradient on tcgen05
// The same convolution as an implicit GEMM on the 5th-generation tensor
// cores, with the M dimension running over the pixels of the zero-padded
// image (rows of W + 2: one zero column on each side; the two padding
// outputs of each row are computed and dropped).  In that indexing the
// three horizontal taps of one row offset dy read the same 130 consecutive
// padded pixels, shifted by 0, 1, 2: a CTA stages one such band per
// (dy, 32-channel block) with cp.async (zero-filled outside the image) and
// issues 3 taps x 2 (K = 16) tcgen05.mma (kind::f16, bf16 x bf16 -> f32)
// from it, the tap shift being a 16-byte offset of the operand's start
// address.  The weights come pre-packed in that operand layout (one
// contiguous run of BN rows per tap and K group), fetched by one thread as
// 12 bulk copies per stage completing on the stage's weight mbarrier.
// Operands sit in the no-swizzle K-major canonical layout: rows of 8
// channels (16 B) consecutive within a K group, 8-row groups 128 B apart
// (SBO), K groups one band (or one weight tile) apart (LBO).  One
// thread issues the MMAs and commits each stage to its mbarrier, which
// releases the stage for the next refill; the 128 x BN f32 accumulator
// lives in tensor memory (BN columns per CTA) and the epilogue reads it
// with tcgen05.ld, one pixel per thread.  Every wait is bounded (the
// kernel then records NLH_ERR_TIMEOUT, skips its stores and still frees
// its tensor memory).
// Two stages (load of chunk k + 1 overlapping the MMAs of chunk k): the
// small footprint keeps 3 (BN 128) to 7 (BN 32) CTAs on an SM, which hides
// the load latency better than a deeper pipeline with fewer CTAs (measured:
// 2 stages 1.23 ms, 3 stages 1.35 ms, 4 stages 1.78 ms for the forward pass
// of 16 images of 256 x 256).
constexpr int kTcStages = 2;
constexpr int kBandRows = kBM + 2;  // 128 outputs + one halo pixel each side

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < kMbarSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bytes of one pipeline stage: the band (4 K groups of 130 rows) and the
// three taps' weight tiles (each 4 K groups of BN rows).
template <int BN> struct TcTile {
    static constexpr int A_BYTES = 4 * kBandRows * 16;  // 8320
    static constexpr int B_TAP = BN * kBK * 2;
    static constexpr int STAGE = A_BYTES + 3 * B_TAP;
    static constexpr int SMEM = kTcStages * STAGE + 128;
};

template <int BN>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3x3_tc(ConvArgs a, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    using T = TcTile<BN>;
    constexpr uint32_t KA = kBandRows * 16, KB = (BN / 8) * 128;  // K-group strides
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(kBM >> 4) << 24);
    // bars: MMA commits per stage; wbars: weight bulk copies per stage
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTcStages * T::STAGE);
    uint64_t *wbars = bars + kTcStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(wbars + kTcStages);
    int *s_fail = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Wp = a.W + 2;
    const int64_t Pp = (int64_t)a.B * a.H * Wp;  // padded pixels
    const int64_t q0 = (int64_t)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const int cin = a.src.c1 + a.src.c2;
    const int kcb = cin / kBK;
    const int nk = 3 * kcb;  // chunks: (band dy, channel block)

    if (tid == 0) {
        for (int st = 0; st < kTcStages; ++st) {
            mbar_init(bars + st, 1);
            mbar_init(wbars + st, 1);
        }
        mbar_fence_init();
        *s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // band rows of this thread: i = tid and (tid < 2) i = 128 + tid; row i
    // holds the padded pixel q0 - 1 + i shifted by the band's dy
    int rb[2], ry[2], rx[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t sidx = q0 - 1 + tid + h * kBM;
        rb[h] = -1;
        if (sidx >= 0 && sidx < Pp && (h == 0 || tid < 2)) {
            const int64_t r = sidx / Wp;
            const int xp = (int)(sidx - r * Wp);
            rb[h] = (int)(r / a.H);
            ry[h] = (int)(r - (int64_t)rb[h] * a.H);
            rx[h] = xp - 1;  // -1 and W are the padding columns
        }
    }
    int w_issued = 0;  // thread 0: chunks whose weight copies were issued
    auto load = [&](int stage, int kc) {
        const int band = kc / kcb, cb = kc - band * kcb;
        const int dy = band - 1;  // input row offset of the band
        const int c0 = cb * kBK;
        const uint32_t sa = smem_u32(smem + stage * T::STAGE);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && tid >= 2) break;
            const int i = tid + h * kBM;
            const bf16 *p = rb[h] >= 0 ? src_ptr(a.src, rb[h], ry[h] + dy, rx[h], a.H, a.W, c0)
                                       : nullptr;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cp_async16(sa + q * KA + i * 16, p ? p + 8 * q : a.w, p != nullptr);
        }
        // weights of the band's three taps (input offset (dy, dx) is tap
        // (sign dy + 1) * 3 + (sign dx + 1)): the packed layout holds each
        // (tap, channel block, K group) as n rows of 16 B, so the BN rows
        // of this CTA are one contiguous bulk copy, 12 per chunk
        if (tid == 0) {
            ++w_issued;
            unsigned char *dst = smem + stage * T::STAGE + T::A_BYTES;
            mbar_arrive_expect_tx(wbars + stage, 12u * BN * 16u);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int tap = (a.sign * dy + 1) * 3 + (a.sign * (t - 1) + 1);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bf16 *wp = a.wt + ((((int64_t)tap * kcb + cb) * 4 + q) * a.n + n0) * 8;
                    bulk_copy_g2s(dst + t * T::B_TAP + q * KB, wp, BN * 16, wbars + stage);
                }
            }
        }
    };

    bool ok = true;
    int w_waited = 0;  // thread 0: chunks whose weight copies have landed
#pragma unroll
    for (int st = 0; st < kTcStages - 1; ++st) {
        if (st < nk) load(st, st);
        cp_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        const int stage = kc % kTcStages;
        cp_wait<kTcStages - 2>();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && ok) {
            if (tc_wait(wbars + stage, (kc / kTcStages) & 1))
                w_waited = kc + 1;
            else
                ok = false;
        }
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + stage * T::STAGE);
            const uint32_t sb = sa + T::A_BYTES;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    // output row m reads band row m + t (tap dx = t - 1)
                    const uint64_t da = tc_desc(sa + ks * 2 * KA + t * 16, KA, 128);
                    const uint64_t db = tc_desc(sb + t * T::B_TAP + ks * 2 * KB, KB, 128);
                    const uint32_t acc = (kc > 0 || t > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(IDESC), "r"(acc));
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(bars + stage))
                : "memory");
        }
        // refill the stage of chunk kc - 1 once its MMAs have read it
        const int nx = kc + kTcStages - 1;
        if (nx < nk) {
            if (kc >= 1 && ok) {
                const int c = kc - 1;
                if (!tc_wait(bars + (c % kTcStages), (c / kTcStages) & 1)) ok = false;
            }
            if (ok) load(nx % kTcStages, nx);
        }
        cp_commit();
    }
    cp_wait<0>();
    // drain: the commits not yet waited for (the last chunk's covers every
    // MMA issued before it; the others are consumed so no arrival is left)
    for (int c = nk - kTcStages > 0 ? nk - kTcStages : 0; c < nk && ok; ++c)
        if (!tc_wait(bars + (c % kTcStages), (c / kTcStages) & 1)) ok = false;
    if (tid == 0 && !ok) {
        // after a failed wait: let the weight copies still in flight land
        // (bounded) before the shared memory is released
        for (int c = w_waited; c < w_issued; ++c)
            if (!tc_wait(wbars + (c % kTcStages), (c / kTcStages) & 1)) break;
    }
    if (!ok) atomicExch(s_fail, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool failed = *s_fail != 0;
    if (failed && tid == 0 && err) atomicExch(err, (int)NLH_ERR_TIMEOUT);

    // epilogue: accumulator row (= padded pixel q0 + 32 warp + lane) per thread
    const int64_t qm = q0 + warp * 32 + lane;
    int64_t mm = -1;  // unpadded output pixel, or -1 (padding column / past the end)
    if (qm < Pp) {
        const int64_t r = qm / Wp;
        const int xp = (int)(qm - r * Wp);
        if (xp >= 1 && xp <= a.W) mm = r * a.W + (xp - 1);
    }
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (failed || mm < 0) continue;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = __uint_as_float(r[j]);
            if (a.bias) v[j] += a.bias[n0 + c0 + j];
            if (a.relu) v[j] = fmaxf(v[j], 0.f);
        }
        const int n = n0 + c0;
        if (a.ybf) {
            __align__(16) bf16 o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16_rn(v[j]);
            uint4 *dst = reinterpret_cast<uint4 *>(a.ybf + mm * a.n + n);
            dst[0] = reinterpret_cast<const uint4 *>(o)[0];
            dst[1] = reinterpret_cast<const uint4 *>(o)[1];
        } else {
            float *dst = n < a.n1 ? a.y1 + mm * a.n1 + n : a.y2 + mm * (a.n - a.n1) + (n - a.n1);
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ----------------------------------------------------------- weight gradient
struct WgradArgs {
    Src src;            // the forward input of the layer
    const bf16 *dz;     // [P][n] gradient at the pre-activation
    int B, H, W;
    int n;              // output channels of the layer
    int cin_real;       // canonical input channels (first layer: 3)
    float *dw;          // canonical gradient W[n][3][3][cin_real], accumulated
    int64_t pix_per_split;
};

// grid: x = pixel split, y = tap * (cin / 32) + channel block, z = block of
// BMW output channels; BMW / 16 warps, each 16 output channels x 32 inputs.
template <int BMW>
__global__ void __launch_bounds__(BMW * 2) k_conv3x3_wgrad(WgradArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NT = BMW * 2;
    constexpr int CPRA = BMW / 8;
    constexpr int A_BYTES = 32 * BMW * 2;
    constexpr int B_BYTES = 32 * 32 * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cin = a.src.c1 + a.src.c2;
    const int kcb = cin / 32;
    const int tap = blockIdx.y / kcb, cb = blockIdx.y - (blockIdx.y / kcb) * kcb;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int c0 = cb * 32;
    const int co0 = blockIdx.z * BMW;
    const int HW = a.H * a.W;
    const int64_t P = (int64_t)a.B * HW;
    const int64_t pbeg = (int64_t)blockIdx.x * a.pix_per_split;
    const int64_t pend = P < pbeg + a.pix_per_split ? P : pbeg + a.pix_per_split;
    const int nch = pbeg < pend ? (int)((pend - pbeg + 31) / 32) : 0;

    auto load = [&](int stage, int kc) {
        const int64_t p0 = pbeg + (int64_t)kc * 32;
        const uint32_t sa = smem_u32(smem + stage * STAGE);
        const uint32_t sb = sa + A_BYTES;
#pragma unroll
        for (int i = 0; i < 32 * CPRA / NT; ++i) {
            const int idx = tid + i * NT;
            const int r = idx / CPRA, q = idx - (idx / CPRA) * CPRA;
            const int64_t p = p0 + r;
            const bool ok = p < pend;
            cp_async16(sa + (r * CPRA + swz<CPRA>(r, q)) * 16,
                       ok ? a.dz + p * a.n + co0 + 8 * q : a.dz, ok);
        }
#pragma unroll
        for (int i = 0; i < 128 / NT; ++i) {
            const int idx = tid + i * NT;
            const int r = idx >> 2, q = idx & 3;
            const int64_t p = p0 + r;
            const bf16 *src = nullptr;
            if (p < pend) {
                const int b = (int)(p / HW);
                const int rem = (int)(p - (int64_t)b * HW);
                const int y = rem / a.W, x = rem - (rem / a.W) * a.W;
                src = src_ptr(a.src, b, y + dy, x + dx, a.H, a.W, c0);
            }
            cp_async16(sb + (r * 4 + swz<4>(r, q)) * 16, src ? src + 8 * q : a.dz,
                       src != nullptr);
        }
    };

    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nch) load(s, s);
        cp_commit();
    }
    for (int kc = 0; kc < nch; ++kc) {
        cp_wait<kStages - 2>();
        __syncthreads();
        {
            const int nx = kc + kStages - 1;
            if (nx < nch) load(nx % kStages, nx);
            cp_commit();
        }
        const uint32_t sa = smem_u32(smem + (kc % kStages) * STAGE);
        const uint32_t sb = sa + A_BYTES;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t af[4];
            {
                const int row = ks * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int ch = warp * 2 + ((lane >> 3) & 1);
                ldsm_x4_t(sa + (row * CPRA + swz<CPRA>(row, ch)) * 16, af[0], af[1], af[2],
                          af[3]);
            }
#pragma unroll
            for (int jb = 0; jb < 2; ++jb) {
                const int row = ks * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);
                const int ch = jb * 2 + (lane >> 4);
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(sb + (row * 4 + swz<4>(row, ch)) * 16, b0, b1, b2, b3);
                mma_bf16(acc[2 * jb], af, b0, b1);
                mma_bf16(acc[2 * jb + 1], af, b2, b3);
            }
        }
    }
    cp_wait<0>();
    if (nch == 0) return;

    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int co = co0 + warp * 16 + g + (e >> 1) * 8;
            const int ci = c0 + j * 8 + 2 * t + (e & 1);
            if (ci < a.cin_real)
                atomicAdd(a.dw + ((int64_t)co * 9 + tap) * a.cin_real + ci, acc[j][e]);
        }
}

// Weight gradient on tcgen05.  dW[co][tap][ci] = sum_p dZ[p][co] X[p + off][ci]
// as a GEMM with M = output channels (MT = 64 or 128 per CTA), N = 32 input
// channels, K = pixels, both operands read MN-major (idesc transpose bits):
// A = dZ as planes of 8 channels [co / 8][pixel][8], B = the same 130-pixel
// band of the input as the forward kernel ([ci / 8][band row][8]), so that
// the three horizontal taps of the CTA's row offset dy are the band shifted
// by 0, 1, 2 rows (16-byte steps of the start address).  K runs over the
// zero-padded image's pixels, 128 per chunk (dZ is zero-filled at the
// padding).  Three accumulators (one per tap, 32 columns each) in tensor
// memory; after the CTA's chunks the epilogue adds them to the canonical
// gradient with f32 atomics (split K).  With MT = 64 the accumulator row r
// sits in lane (r / 16) 32 + r % 16.  Descriptors: LBO = stride between
// K-direction core matrices (128 B), SBO = stride between M/N-direction
// ones (one plane).  Grid: x = pixel split, y = (input block) * 3 + dy + 1,
// z = block of MT output channels.
constexpr int kWgChunk = 128;  // padded pixels per K chunk

template <int MT> struct WgTile {
    static constexpr int A_BYTES = MT * kWgChunk * 2;
    static constexpr int B_BYTES = 4 * kBandRows * 16;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = kTcStages * STAGE + 128;
};

template <int MT>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3x3_wgrad_tc(WgradArgs a, int n_chunks,
                                                                      int chunks_per_split,
                                                                      int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    using T = WgTile<MT>;
    constexpr uint32_t SBO_A = kWgChunk * 16, SBO_B = kBandRows * 16;
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
    const int ch0 = blockIdx.x * chunks_per_split;
    const int nch = min(n_chunks, ch0 + chunks_per_split) - ch0;
    if (nch <= 0) return;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTcStages * T::STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kTcStages);
    int *s_fail = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Wp = a.W + 2;
    const int64_t Pp = (int64_t)a.B * a.H * Wp;
    const int cb = blockIdx.y / 3, dy = (int)(blockIdx.y % 3) - 1;
    const int c0 = cb * 32;
    const int co0 = blockIdx.z * MT;
    const int co_groups = min(MT, a.n - co0) / 8;  // loaded planes; the rest stay zero

    // zero both stages once (planes beyond the layer's channels stay zero)
    for (int i = tid; i < kTcStages * T::STAGE / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int st = 0; st < kTcStages; ++st) mbar_init(bars + st, 1);
        mbar_fence_init();
        *s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
            smem_u32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    auto load = [&](int stage, int c) {
        const int64_t q0 = (int64_t)(ch0 + c) * kWgChunk;
        const uint32_t sa = smem_u32(smem + stage * T::STAGE);
        const uint32_t sb = sa + T::A_BYTES;
        // A: dZ of padded pixel q0 + tid (zero at the padding and past the end)
        {
            const int64_t q = q0 + tid;
            const bf16 *p = nullptr;
            if (q < Pp) {
                const int64_t r = q / Wp;
                const int xp = (int)(q - r * Wp);
                if (xp >= 1 && xp <= a.W) p = a.dz + (r * a.W + (xp - 1)) * a.n + co0;
            }
            for (int g = 0; g < co_groups; ++g)
                cp_async16(sa + g * SBO_A + tid * 16, p ? p + 8 * g : a.dz, p != nullptr);
        }
        // B: band rows i = tid and (tid < 2) 128 + tid: padded pixel
        // q0 - 1 + i shifted by dy rows
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && tid >= 2) break;
            const int i = tid + h * kConvThreads;
            const int64_t sidx = q0 - 1 + i;
            const bf16 *p = nullptr;
            if (sidx >= 0 && sidx < Pp) {
                const int64_t r = sidx / Wp;
                const int xp = (int)(sidx - r * Wp);
                const int b = (int)(r / a.H), y = (int)(r - (int64_t)b * a.H);
                p = src_ptr(a.src, b, y + dy, xp - 1, a.H, a.W, c0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cp_async16(sb + q * SBO_B + i * 16, p ? p + 8 * q : a.dz, p != nullptr);
        }
    };

    bool ok = true;
#pragma unroll
    for (int st = 0; st < kTcStages - 1; ++st) {
        if (st < nch) load(st, st);
        cp_commit();
    }
    for (int c = 0; c < nch; ++c) {
        const int stage = c % kTcStages;
        cp_wait<kTcStages - 2>();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + stage * T::STAGE);
            const uint32_t sb = sa + T::A_BYTES;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
#pragma unroll
                for (int ks = 0; ks < kWgChunk / 16; ++ks) {
                    // tap dx = t - 1 reads band row k + t for pixel k
                    const uint64_t da = tc_desc(sa + ks * 256, 128, SBO_A);
                    const uint64_t db = tc_desc(sb + t * 16 + ks * 256, 128, SBO_B);
                    const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                            tmem + (uint32_t)(t * 32)),
                        "l"(da), "l"(db), "r"(IDESC), "r"(acc));
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(bars + stage))
                : "memory");
        }
        // refill the stage of chunk c - 1 once its MMAs have read it
        const int nx = c + kTcStages - 1;
        if (nx < nch) {
            if (c >= 1 && ok) {
                const int w = c - 1;
                if (!tc_wait(bars + (w % kTcStages), (w / kTcStages) & 1)) ok = false;
            }
            if (ok) load(nx % kTcStages, nx);
        }
        cp_commit();
    }
    cp_wait<0>();
    for (int w = nch - kTcStages > 0 ? nch - kTcStages : 0; w < nch && ok; ++w)
        if (!tc_wait(bars + (w % kTcStages), (w / kTcStages) & 1)) ok = false;
    if (!ok) atomicExch(s_fail, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool failed = *s_fail != 0;
    if (failed && tid == 0 && err) atomicExch(err, (int)NLH_ERR_TIMEOUT);

    // epilogue: accumulator row of this lane (MT = 64: lanes 0..15 of each warp)
    const int row = MT == 128 ? warp * 32 + lane : (lane < 16 ? warp * 16 + lane : -1);
    const int co = co0 + row;
    const bool live = !failed && row >= 0 && co < a.n;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int tap = (dy + 1) * 3 + t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r[16];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 32 + h * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!live) continue;
            float *dst = a.dw + ((int64_t)co * 9 + tap) * a.cin_real;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int ci = c0 + h * 16 + j;
                if (ci < a.cin_real) atomicAdd(dst + ci, __uint_as_float(r[j]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// ------------------------------------------------------ elementwise kernels
struct Scalars {
    float ls[kMaxBatch], la[kMaxBatch];  // ln sigma, ln alpha per image
    double alpha[kMaxBatch];
};

// x0[p] = [f, ln sigma, ln alpha, 0 x 29] (bf16, 32 channels)
__global__ void k_input_planes(const double *__restrict__ f, int64_t P, int HW, Scalars sc,
                               bf16 *__restrict__ x0) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(p / HW);
        __align__(16) bf16 v[8];
        v[0] = __float2bfloat16_rn((float)f[p]);
        v[1] = __float2bfloat16_rn(sc.ls[b]);
        v[2] = __float2bfloat16_rn(sc.la[b]);
#pragma unroll
        for (int k = 3; k < 8; ++k) v[k] = __float2bfloat16_rn(0.f);
        uint4 *dst = reinterpret_cast<uint4 *>(x0 + p * 32);
        dst[0] = *reinterpret_cast<const uint4 *>(v);
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        dst[1] = z;
        dst[2] = z;
        dst[3] = z;
    }
}

// 2x2 average pooling, bf16 -> bf16 (sum in f32).  H, W of the input.
__global__ void k_avgpool2(const bf16 *__restrict__ x, int B, int H, int W, int C,
                           bf16 *__restrict__ y) {
    const int Ho = H / 2, Wo = W / 2, G = C / 8;
    const int64_t total = (int64_t)B * Ho * Wo * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int cg = (int)(i % G);
        const int64_t q = i / G;
        const int xo = (int)(q % Wo);
        const int64_t r = q / Wo;
        const int yo = (int)(r % Ho);
        const int b = (int)(r / Ho);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int yy = 2 * yo + (d >> 1), xx = 2 * xo + (d & 1);
            const uint4 raw = *reinterpret_cast<const uint4 *>(
                x + (((int64_t)b * H + yy) * W + xx) * C + cg * 8);
            const bf16 *v = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(v[k]);
        }
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16_rn(0.25f * s[k]);
        *reinterpret_cast<uint4 *>(y + q * C + cg * 8) = *reinterpret_cast<const uint4 *>(o);
    }
}

// The gradient at a ReLU output y (level of size B x H x W, C channels):
//   g = same[p] + coarse[parent(p)] / 4 + sum over the 4 children of fine,
// dz = g * (y > 0) in bf16, db[c] += sum_p dz (f32, before rounding).
// Each thread keeps one 8-channel group (the grid's thread count is a
// multiple of C / 8), so the bias partials stay in registers.
__global__ void __launch_bounds__(kElemThreads)
k_grad_merge(const float *__restrict__ same, const float *__restrict__ coarse,
             const float *__restrict__ fine, const bf16 *__restrict__ y, int B, int H, int W,
             int C, bf16 *__restrict__ dz, float *__restrict__ db) {
    __shared__ float red[kElemThreads][9];
    const int G = C / 8;
    const int64_t P = (int64_t)B * H * W;
    const int64_t total = P * G;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int cg = (int)(gt % G);
    float bs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = gt; i < total; i += stride) {
        const int64_t p = i / G;
        float g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (same) {
            const float4 *s4 = reinterpret_cast<const float4 *>(same + p * C + cg * 8);
            const float4 u = s4[0], v = s4[1];
            g[0] = u.x, g[1] = u.y, g[2] = u.z, g[3] = u.w;
            g[4] = v.x, g[5] = v.y, g[6] = v.z, g[7] = v.w;
        }
        if (coarse || fine) {
            const int x = (int)(p % W);
            const int64_t r = p / W;
            const int yy = (int)(r % H);
            const int b = (int)(r / H);
            if (coarse) {
                const float4 *s4 = reinterpret_cast<const float4 *>(
                    coarse + (((int64_t)b * (H / 2) + yy / 2) * (W / 2) + x / 2) * C + cg * 8);
                const float4 u = s4[0], v = s4[1];
                g[0] += 0.25f * u.x, g[1] += 0.25f * u.y, g[2] += 0.25f * u.z, g[3] += 0.25f * u.w;
                g[4] += 0.25f * v.x, g[5] += 0.25f * v.y, g[6] += 0.25f * v.z, g[7] += 0.25f * v.w;
            }
            if (fine) {
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    const float4 *s4 = reinterpret_cast<const float4 *>(
                        fine +
                        (((int64_t)b * (2 * H) + 2 * yy + (d >> 1)) * (2 * W) + 2 * x + (d & 1)) *
                            C +
                        cg * 8);
                    const float4 u = s4[0], v = s4[1];
                    g[0] += u.x, g[1] += u.y, g[2] += u.z, g[3] += u.w;
                    g[4] += v.x, g[5] += v.y, g[6] += v.z, g[7] += v.w;
                }
            }
        }
        const uint4 raw = *reinterpret_cast<const uint4 *>(y + p * C + cg * 8);
        const bf16 *yv = reinterpret_cast<const bf16 *>(&raw);
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float v = __bfloat162float(yv[k]) > 0.f ? g[k] : 0.f;
            bs[k] += v;
            o[k] = __float2bfloat16_rn(v);
        }
        *reinterpret_cast<uint4 *>(dz + p * C + cg * 8) = *reinterpret_cast<const uint4 *>(o);
    }
    // bias gradient: threads of the block with the same channel group
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = bs[k];
    __syncthreads();
    // the channel group of thread t is (blockIdx.x * blockDim.x + t) % G
    if (threadIdx.x < G) {
        const int my = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % G);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = threadIdx.x; t < kElemThreads; t += G)
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += red[t][k];
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(db + my * 8 + k, s[k]);
    }
}

// Head: o[p] = Wh d0[p] + bh (f32); u0 = mean(f of the image) + o0,
// scale = exp(clamp(o1, -4, 4)).  stats[3 b] is the mean of image b.
template <int C>
__global__ void k_head_fwd(const bf16 *__restrict__ d0, int64_t P, int HW,
                           const float *__restrict__ wh, const double *__restrict__ stats,
                           float2 *__restrict__ o, double *__restrict__ u0,
                           double *__restrict__ scale) {
    __shared__ float w[2 * C + 2];
    for (int k = threadIdx.x; k < 2 * C + 2; k += blockDim.x) w[k] = wh[k];
    __syncthreads();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        float o0 = w[2 * C], o1 = w[2 * C + 1];
#pragma unroll
        for (int cg = 0; cg < C / 8; ++cg) {
            const uint4 raw = *reinterpret_cast<const uint4 *>(d0 + p * C + cg * 8);
            const bf16 *v = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float x = __bfloat162float(v[k]);
                o0 = fmaf(w[cg * 8 + k], x, o0);
                o1 = fmaf(w[C + cg * 8 + k], x, o1);
            }
        }
        if (o) o[p] = make_float2(o0, o1);
        if (u0) u0[p] = stats[3 * (p / HW)] + (double)o0;
        if (scale) scale[p] = exp((double)fminf(fmaxf(o1, -4.f), 4.f));
    }
}

// Per image b: stats[3b] = mean(f), stats[3b+1] = ||alpha (f - mean f)||^2
// (the residual of the deflated start), stats[3b+2] = ||e0||^2.
__device__ __forceinline__ double block_sum_d(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Partial sums of image b over the slice blockIdx.x of gridDim.x:
// part[3 (b G + g) + {0, 1, 2}] = sum (f - K), sum (f - K)^2, sum e0^2, with
// the shift K = f[b][0] (so that the variance below does not cancel).
constexpr int kStatsMaxSlices = 64;
__global__ void __launch_bounds__(kElemThreads)
k_stats_partial(const double *__restrict__ f, const double *__restrict__ e0, int HW,
                double *__restrict__ part) {
    __shared__ double sh[kElemThreads];
    const int b = blockIdx.y, G = gridDim.x;
    const double *fb = f + (int64_t)b * HW;
    const double K = fb[0];
    double s1 = 0.0, s2 = 0.0, se = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += G * blockDim.x) {
        const double d = fb[i] - K;
        s1 += d;
        s2 = fma(d, d, s2);
        if (e0) se = fma(e0[(int64_t)b * HW + i], e0[(int64_t)b * HW + i], se);
    }
    s1 = block_sum_d(s1, sh);
    s2 = block_sum_d(s2, sh);
    se = block_sum_d(se, sh);
    if (threadIdx.x == 0) {
        double *o = part + 3 * ((int64_t)b * G + blockIdx.x);
        o[0] = s1, o[1] = s2, o[2] = se;
    }
}

// One block per image sums the G partials in a fixed order:
// stats[3b] = mean(f) = K + S1 / HW,
// stats[3b+1] = ||alpha (f - mean f)||^2 = alpha^2 (S2 - S1^2 / HW),
// stats[3b+2] = ||e0||^2 (the residual of the deflated start and the norm
// of the preconditioner term's target).
__global__ void k_stats_final(const double *__restrict__ f, const double *__restrict__ part, int G,
                              int HW, Scalars sc, double *__restrict__ stats) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s1 = 0.0, s2 = 0.0, se = 0.0;
    for (int g = 0; g < G; ++g) {
        const double *o = part + 3 * ((int64_t)b * G + g);
        s1 += o[0], s2 += o[1], se += o[2];
    }
    const double mean = f[(int64_t)b * HW] + s1 / HW;
    const double nu = sc.alpha[b] * sc.alpha[b] * (s2 - s1 * s1 / HW);
    stats[3 * b] = mean;
    stats[3 * b + 1] = nu > 0.0 ? nu : 1e-300;
    stats[3 * b + 2] = se > 0.0 ? se : 1e-300;
}

// Loss and its gradient with respect to the head outputs (see nlh_net.h).
__global__ void __launch_bounds__(kElemThreads)
k_loss_grad(const float2 *__restrict__ o, const double *__restrict__ us,
            const double *__restrict__ r0, const double *__restrict__ e0,
            const double *__restrict__ deg, const double *__restrict__ stats, Scalars sc, int B,
            int HW, double beta, float2 *__restrict__ dout, double *__restrict__ loss) {
    __shared__ double red[kElemThreads];
    const int64_t P = (int64_t)B * HW;
    const double inv_b = 1.0 / B;
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(p / HW);
        const float2 op = o[p];
        const double pa = sc.alpha[b] + fmax(deg[p] - 1.0, 0.0);
        const double du = stats[3 * b] + (double)op.x - us[p];
        const double nu = stats[3 * b + 1];
        acc += pa * pa * du * du / nu;
        const double g0 = 2.0 * inv_b * pa * pa * du / nu;
        double g1 = 0.0;
        if (beta > 0.0) {
            const double ne = stats[3 * b + 2];
            const double c = (double)fminf(fmaxf(op.y, -4.f), 4.f);
            const double pr = r0[p] / (pa * exp(c));
            const double dl = pr - e0[p];
            acc += beta * dl * dl / ne;
            if (op.y > -4.f && op.y < 4.f) g1 = -2.0 * inv_b * beta * dl * pr / ne;
        }
        dout[p] = make_float2((float)g0, (float)g1);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_b);
}

// Head backward: dd0[p][c] = sum_j Wh[j][c] dout[p][j]; dWh, dbh reduced
// over pixels (registers, then warp shuffles, then shared memory, then one
// atomic per value per block).
template <int C>
__global__ void __launch_bounds__(kElemThreads)
k_head_bwd(const bf16 *__restrict__ d0, const float2 *__restrict__ dout, int64_t P,
           const float *__restrict__ wh, float *__restrict__ dd0, float *__restrict__ gwh) {
    __shared__ float w[2 * C];
    __shared__ float red[kElemThreads / 32][2 * C + 2];
    for (int k = threadIdx.x; k < 2 * C; k += blockDim.x) w[k] = wh[k];
    __syncthreads();
    float gw[2 * C + 2];
#pragma unroll
    for (int k = 0; k < 2 * C + 2; ++k) gw[k] = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float2 g = dout[p];
#pragma unroll
        for (int cg = 0; cg < C / 8; ++cg) {
            const uint4 raw = *reinterpret_cast<const uint4 *>(d0 + p * C + cg * 8);
            const bf16 *v = reinterpret_cast<const bf16 *>(&raw);
            float od[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float x = __bfloat162float(v[k]);
                const int c = cg * 8 + k;
                gw[c] = fmaf(g.x, x, gw[c]);
                gw[C + c] = fmaf(g.y, x, gw[C + c]);
                od[k] = w[c] * g.x + w[C + c] * g.y;
            }
            float4 *dst = reinterpret_cast<float4 *>(dd0 + p * C + cg * 8);
            dst[0] = make_float4(od[0], od[1], od[2], od[3]);
            dst[1] = make_float4(od[4], od[5], od[6], od[7]);
        }
        gw[2 * C] += g.x;
        gw[2 * C + 1] += g.y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * C + 2; ++k) {
        float v = gw[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * C + 2; k += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < kElemThreads / 32; ++q) s += red[q][k];
        atomicAdd(gwh + k, s);
    }
}

// (1 - b1) and (1 - b2) come in separately, formed in FP64, so that the
// moment scaling and the bias correction 1 / (1 - b^t) agree to FP32
// rounding (1 - 0.9f in FP32 is 0.100000024).
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1,
                       float omb1, float b2, float omb2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + omb1 * gi;
        const float vi = b2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

struct PackTable {
    int nl;
    int cin[16], cinp[16], cout[16];
    int64_t woff[16], wfoff[16], wdoff[16], start[17];
};

// theta -> Wf[cout][9][cinp] and Wd[cinp][9][cout] (bf16; zero padding),
// and both again in the tcgen05 layout.
// The tcgen05 engine's copies: a GEMM weight w[n][9][k] (forward: n =
// cout, k = cinp; input gradient: n = cinp, k = cout) as
// [9][k / 32][4][n][8], element (n, tap, kk) at
// ((tap (k / 32) + kk / 32) 4 + (kk % 32) / 8) n 8 + n 8 + kk % 8.
__device__ __forceinline__ int64_t tc_pack_index(int n, int tap, int kk, int N, int K) {
    return (((int64_t)tap * (K / 32) + kk / 32) * 4 + (kk % 32) / 8) * N * 8 + (int64_t)n * 8 +
           kk % 8;
}

__global__ void k_pack_weights(const float *__restrict__ theta, PackTable t, bf16 *__restrict__ wf,
                               bf16 *__restrict__ wd, bf16 *__restrict__ wtf,
                               bf16 *__restrict__ wtd) {
    const int64_t total = t.start[t.nl];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (i >= t.start[l + 1]) ++l;
        const int64_t loc = i - t.start[l];
        const int cinp = t.cinp[l];
        const int co = (int)(loc / (9 * cinp));
        const int rem = (int)(loc - (int64_t)co * 9 * cinp);
        const int tap = rem / cinp, ci = rem - (rem / cinp) * cinp;
        const float val =
            ci < t.cin[l] ? theta[t.woff[l] + ((int64_t)co * 9 + tap) * t.cin[l] + ci] : 0.f;
        const bf16 b = __float2bfloat16_rn(val);
        wf[t.wfoff[l] + loc] = b;
        wd[t.wdoff[l] + ((int64_t)ci * 9 + tap) * t.cout[l] + co] = b;
        wtf[t.wfoff[l] + tc_pack_index(co, tap, ci, t.cout[l], cinp)] = b;
        wtd[t.wdoff[l] + tc_pack_index(ci, tap, co, cinp, t.cout[l])] = b;
    }
}

// e0 = us - u0
// (u0 and e0 may be the same array)
__global__ void k_sub(const double *us, const double *u0, int64_t n, double *e0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        e0[i] = us[i] - u0[i];
}

}  // namespace netk
}  // namespace nlh

// ====================================================================== host
using namespace nlh;
using netk::bf16;

namespace {

constexpr int kSMs = 152;

struct LayerDesc {
    int cin, cout, k, cinp;
    int64_t woff, boff, wfoff, wdoff;
};

struct Level {
    bf16 *Q = nullptr, *A = nullptr, *E = nullptr, *DA = nullptr, *D = nullptr;
    float *S = nullptr;
};

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8 * kSMs));
}

}  // namespace

struct nlh_net_s {
    int base = 32, levels = 4;
    std::vector<LayerDesc> layers;  // 3x3 layers then the head
    int64_t n_params = 0, wf_total = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf = nullptr, *wd = nullptr, *wtf = nullptr, *wtd = nullptr;
    bool packed = false;
    int adam_t = 0;
    int engine = NLH_NET_ENGINE_TCGEN05;
    int *err = nullptr;  // device error word of the bounded tensor-core waits
    // workspace of the current batch shape
    int B = 0, H = 0, W = 0;
    bool has_grad_ws = false;
    bf16 *X0 = nullptr, *dz = nullptr;
    std::vector<Level> lv;
    float2 *o = nullptr, *dout = nullptr;
    float *T1 = nullptr, *T2 = nullptr;
    double *stats = nullptr, *stats_part = nullptr, *loss = nullptr;
    std::vector<void *> ws;
    netk::PackTable pack{};

    ~nlh_net_s() {
        cudaDeviceSynchronize();
        free_ws();
        cudaFree(theta);
        cudaFree(grad);
        cudaFree(m);
        cudaFree(v);
        cudaFree(wf);
        cudaFree(wd);
        cudaFree(wtf);
        cudaFree(wtd);
        cudaFree(err);
    }
    void free_ws() {
        for (void *p : ws) cudaFree(p);
        ws.clear();
        lv.clear();
        B = H = W = 0;
        has_grad_ws = false;
    }
    template <typename T> T *wsalloc(size_t count) {
        void *p = nullptr;
        NLH_CUDA(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
        ws.push_back(p);
        return (T *)p;
    }
    int ch(int l) const { return base << l; }
    int index(bool enc, int l, int ab) const {
        // enc: 2l + ab; dec (levels-2 .. 0): 2 levels + 2 (levels - 2 - l) + ab
        return enc ? 2 * l + ab : 2 * levels + 2 * (levels - 2 - l) + ab;
    }
};

static void net_ensure_ws(nlh_net_s &N, int B, int H, int W, bool grad, cudaStream_t s) {
    if (N.B == B && N.H == H && N.W == W && (N.has_grad_ws || !grad)) return;
    NLH_CUDA(cudaStreamSynchronize(s));
    N.free_ws();
    const int64_t P0 = (int64_t)B * H * W;
    N.X0 = N.wsalloc<bf16>(P0 * 32);
    N.lv.resize(N.levels);
    for (int l = 0; l < N.levels; ++l) {
        const int64_t P = P0 >> (2 * l);
        Level &L = N.lv[l];
        if (l > 0) L.Q = N.wsalloc<bf16>(P * N.ch(l - 1));
        L.A = N.wsalloc<bf16>(P * N.ch(l));
        L.E = N.wsalloc<bf16>(P * N.ch(l));
        if (l < N.levels - 1) {
            L.DA = N.wsalloc<bf16>(P * N.ch(l));
            L.D = N.wsalloc<bf16>(P * N.ch(l));
        }
    }
    N.o = N.wsalloc<float2>(P0);
    N.stats = N.wsalloc<double>(3 * netk::kMaxBatch);
    N.stats_part = N.wsalloc<double>(3 * netk::kMaxBatch * netk::kStatsMaxSlices);
    if (grad) {
        N.dout = N.wsalloc<float2>(P0);
        N.dz = N.wsalloc<bf16>(P0 * N.ch(0));
        N.T1 = N.wsalloc<float>(P0 * N.ch(1));
        N.T2 = N.wsalloc<float>(P0 * N.ch(0));
        for (int l = 0; l < N.levels - 1; ++l)
            N.lv[l].S = N.wsalloc<float>((P0 >> (2 * l)) * N.ch(l));
        N.loss = N.wsalloc<double>(1);
    }
    N.B = B;
    N.H = H;
    N.W = W;
    N.has_grad_ws = grad;
}

static void net_pack(nlh_net_s &N, cudaStream_t s) {
    if (N.packed) return;
    netk::k_pack_weights<<<grid_for(N.wf_total, 256), 256, 0, s>>>(N.theta, N.pack, N.wf, N.wd,
                                                                  N.wtf, N.wtd);
    NLH_CHECK_LAUNCH();
    N.packed = true;
}

// Launch the forward / input-gradient implicit GEMM a with the net's
// engine; BN (output channels per CTA) is the widest of 128, 64, 32 that
// divides n, does not straddle the split n1 and still gives two CTAs per SM.
static void launch_conv(nlh_net_s &N, const netk::ConvArgs &a, int n1, cudaStream_t s) {
    const int64_t P = (int64_t)a.B * a.H * a.W;
    const int mt = (int)((P + netk::kBM - 1) / netk::kBM);
    auto launch = [&](auto bn) {
        constexpr int BN = decltype(bn)::value;
        if (N.engine == NLH_NET_ENGINE_TCGEN05) {
            // M runs over the padded pixels; tensor memory: BN columns per
            // CTA, and the shared-memory footprint keeps at most 512 / BN
            // CTAs on an SM, so allocations never wait
            const int64_t Pp = (int64_t)a.B * a.H * (a.W + 2);
            const int mtp = (int)((Pp + netk::kBM - 1) / netk::kBM);
            const int smem = netk::TcTile<BN>::SMEM;
            NLH_CUDA(cudaFuncSetAttribute(netk::k_conv3x3_tc<BN>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            netk::k_conv3x3_tc<BN><<<dim3(mtp, a.n / BN), netk::kConvThreads, smem, s>>>(a, N.err);
        } else {
            const int smem = netk::kStages * (netk::kBM + BN) * netk::kBK * 2;
            NLH_CUDA(cudaFuncSetAttribute(netk::k_conv3x3<BN>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            netk::k_conv3x3<BN><<<dim3(mt, a.n / BN), netk::kConvThreads, smem, s>>>(a);
        }
        NLH_CHECK_LAUNCH();
    };
    if (a.n % 128 == 0 && n1 % 128 == 0 && (int64_t)mt * (a.n / 128) >= 2 * kSMs)
        launch(std::integral_constant<int, 128>());
    else if (a.n % 64 == 0 && n1 % 64 == 0 && (int64_t)mt * (a.n / 64) >= 2 * kSMs)
        launch(std::integral_constant<int, 64>());
    else
        launch(std::integral_constant<int, 32>());
}

// y = conv3x3(src) with layer li's weights: forward (bias, ReLU, bf16 out).
static void conv_fwd(nlh_net_s &N, int li, netk::Src src, int B, int H, int W, bf16 *y,
                     cudaStream_t s) {
    const LayerDesc &L = N.layers[li];
    NLH_REQUIRE(src.c1 + src.c2 == L.cinp, "net: layer %d input channels", li);
    netk::ConvArgs a{};
    a.src = src;
    a.w = N.wf + L.wfoff;
    a.wt = N.wtf + L.wfoff;
    a.bias = N.theta + L.boff;
    a.relu = 1;
    a.sign = 1;
    a.B = B, a.H = H, a.W = W;
    a.n = L.cout;
    a.ybf = y;
    launch_conv(N, a, 0, s);
}

// Input gradient of layer li: dz [P][cout] -> float [P][cinp], split at n1.
static void conv_dgrad(nlh_net_s &N, int li, const bf16 *dz, int B, int H, int W, float *y1,
                       int n1, float *y2, cudaStream_t s) {
    const LayerDesc &L = N.layers[li];
    netk::ConvArgs a{};
    a.src = netk::Src{dz, L.cout, 0, nullptr, 0};
    a.w = N.wd + L.wdoff;
    a.wt = N.wtd + L.wdoff;
    a.bias = nullptr;
    a.relu = 0;
    a.sign = -1;
    a.B = B, a.H = H, a.W = W;
    a.n = L.cinp;
    a.ybf = nullptr;
    a.y1 = y1;
    a.n1 = n1;
    a.y2 = y2;
    launch_conv(N, a, n1, s);
}

static void conv_wgrad(nlh_net_s &N, int li, netk::Src src, const bf16 *dz, int B, int H, int W,
                       cudaStream_t s) {
    const LayerDesc &L = N.layers[li];
    netk::WgradArgs a{};
    a.src = src;
    a.dz = dz;
    a.B = B, a.H = H, a.W = W;
    a.n = L.cout;
    a.cin_real = L.cin;
    a.dw = N.grad + L.woff;
    if (N.engine == NLH_NET_ENGINE_TCGEN05) {
        // K chunks of 128 padded pixels; about 8 CTAs per SM over the grid,
        // at least 2 chunks per CTA
        const int64_t Pp = (int64_t)B * H * (W + 2);
        const int n_chunks = (int)((Pp + netk::kWgChunk - 1) / netk::kWgChunk);
        const int gy = 3 * (L.cinp / 32);
        auto launch = [&](auto mt) {
            constexpr int MT = decltype(mt)::value;
            const int gz = (L.cout + MT - 1) / MT;
            int64_t splits = (8 * kSMs + (int64_t)gy * gz - 1) / ((int64_t)gy * gz);
            splits = std::max<int64_t>(1, std::min<int64_t>(splits, (n_chunks + 1) / 2));
            const int cps = (int)((n_chunks + splits - 1) / splits);
            splits = (n_chunks + cps - 1) / cps;
            const int smem = netk::WgTile<MT>::SMEM;
            NLH_CUDA(cudaFuncSetAttribute(netk::k_conv3x3_wgrad_tc<MT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            netk::k_conv3x3_wgrad_tc<MT><<<dim3((unsigned)splits, gy, gz), netk::kConvThreads,
                                           smem, s>>>(a, n_chunks, cps, N.err);
            NLH_CHECK_LAUNCH();
        };
        if (L.cout >= 128)
            launch(std::integral_constant<int, 128>());
        else
            launch(std::integral_constant<int, 64>());
        return;
    }
    const int64_t P = (int64_t)B * H * W;
    const int bmw = L.cout % 64 == 0 ? 64 : 32;
    const int gy = 9 * (L.cinp / 32), gz = L.cout / bmw;
    int64_t splits = (4 * kSMs + (int64_t)gy * gz - 1) / ((int64_t)gy * gz);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, (P + 255) / 256));
    int64_t per = (P + splits - 1) / splits;
    per = (per + 31) / 32 * 32;
    splits = (P + per - 1) / per;
    a.pix_per_split = per;
    if (bmw == 64) {
        const int smem = netk::kStages * (32 * 64 + 32 * 32) * 2;
        netk::k_conv3x3_wgrad<64><<<dim3((unsigned)splits, gy, gz), 128, smem, s>>>(a);
    } else {
        const int smem = netk::kStages * (32 * 32 + 32 * 32) * 2;
        netk::k_conv3x3_wgrad<32><<<dim3((unsigned)splits, gy, gz), 64, smem, s>>>(a);
    }
    NLH_CHECK_LAUNCH();
}

static void grad_merge(nlh_net_s &N, int li, const float *same, const float *coarse,
                       const float *fine, const bf16 *y, int B, int H, int W, cudaStream_t s) {
    const LayerDesc &L = N.layers[li];
    const int64_t total = (int64_t)B * H * W * (L.cout / 8);
    netk::k_grad_merge<<<grid_for(total, netk::kElemThreads), netk::kElemThreads, 0, s>>>(
        same, coarse, fine, y, B, H, W, L.cout, N.dz, N.grad + L.boff);
    NLH_CHECK_LAUNCH();
}

static netk::Scalars make_scalars(const nlh_net_batch &b) {
    netk::Scalars sc{};
    for (int i = 0; i < b.B; ++i) {
        NLH_REQUIRE(b.sigma[i] > 0 && b.alpha[i] > 0, "net: sigma and alpha must be > 0");
        sc.ls[i] = (float)std::log(b.sigma[i]);
        sc.la[i] = (float)std::log(b.alpha[i]);
        sc.alpha[i] = b.alpha[i];
    }
    return sc;
}

static void check_batch(const nlh_net_s &N, const nlh_net_batch *b) {
    NLH_REQUIRE(b, "net: batch is NULL");
    const int q = 1 << (N.levels - 1);
    NLH_REQUIRE(b->B >= 1 && b->B <= netk::kMaxBatch, "net: batch size must be in [1, 64]");
    NLH_REQUIRE(b->H >= q && b->W >= q && b->H % q == 0 && b->W % q == 0,
                "net: H and W must be positive multiples of %d", q);
    NLH_REQUIRE(b->f && b->sigma && b->alpha, "net: f, sigma and alpha are required");
}

// Forward pass; keeps every activation in the workspace.
static void net_forward(nlh_net_s &N, const nlh_net_batch &b, double *u0, double *scale,
                        const double *e0_for_stats, cudaStream_t s) {
    net_pack(N, s);
    const int B = b.B, H = b.H, W = b.W;
    const int64_t P0 = (int64_t)B * H * W;
    netk::k_input_planes<<<grid_for(P0, 256), 256, 0, s>>>(b.f, P0, H * W, make_scalars(b), N.X0);
    NLH_CHECK_LAUNCH();
    const bf16 *x = N.X0;
    int cx = 32;
    for (int l = 0; l < N.levels; ++l) {
        const int h = H >> l, w = W >> l;
        Level &L = N.lv[l];
        if (l > 0) {
            const int64_t tot = (int64_t)B * h * w * (cx / 8);
            netk::k_avgpool2<<<grid_for(tot, 256), 256, 0, s>>>(x, B, 2 * h, 2 * w, cx, L.Q);
            NLH_CHECK_LAUNCH();
            x = L.Q;
        }
        conv_fwd(N, N.index(true, l, 0), netk::Src{x, cx, 0, nullptr, 0}, B, h, w, L.A, s);
        conv_fwd(N, N.index(true, l, 1), netk::Src{L.A, N.ch(l), 0, nullptr, 0}, B, h, w, L.E, s);
        x = L.E;
        cx = N.ch(l);
    }
    for (int l = N.levels - 2; l >= 0; --l) {
        const int h = H >> l, w = W >> l;
        Level &L = N.lv[l];
        conv_fwd(N, N.index(false, l, 0), netk::Src{x, cx, 1, L.E, N.ch(l)}, B, h, w, L.DA, s);
        conv_fwd(N, N.index(false, l, 1), netk::Src{L.DA, N.ch(l), 0, nullptr, 0}, B, h, w, L.D,
                 s);
        x = L.D;
        cx = N.ch(l);
    }
    {
        // about two blocks per SM over the batch, at least 2048 pixels each
        const int HW = H * W;
        int G = std::min<int>((2 * kSMs + B - 1) / B, (HW + 2047) / 2048);
        G = std::max(1, std::min(G, netk::kStatsMaxSlices));
        netk::k_stats_partial<<<dim3(G, B), netk::kElemThreads, 0, s>>>(b.f, e0_for_stats, HW,
                                                                        N.stats_part);
        NLH_CHECK_LAUNCH();
        netk::k_stats_final<<<B, 32, 0, s>>>(b.f, N.stats_part, G, HW, make_scalars(b), N.stats);
        NLH_CHECK_LAUNCH();
    }
    const LayerDesc &Hd = N.layers.back();
    if (N.base == 32)
        netk::k_head_fwd<32><<<grid_for(P0, 256), 256, 0, s>>>(x, P0, H * W, N.theta + Hd.woff,
                                                              N.stats, N.o, u0, scale);
    else
        netk::k_head_fwd<64><<<grid_for(P0, 256), 256, 0, s>>>(x, P0, H * W, N.theta + Hd.woff,
                                                              N.stats, N.o, u0, scale);
    NLH_CHECK_LAUNCH();
}

static void net_backward(nlh_net_s &N, const nlh_net_batch &b, cudaStream_t s) {
    const int B = b.B, H = b.H, W = b.W, Lv = N.levels;
    const int64_t P0 = (int64_t)B * H * W;
    NLH_CUDA(cudaMemsetAsync(N.grad, 0, sizeof(float) * N.n_params, s));
    const LayerDesc &Hd = N.layers.back();
    const int gh = std::min(grid_for(P0, netk::kElemThreads), 2 * kSMs);
    if (N.base == 32)
        netk::k_head_bwd<32><<<gh, netk::kElemThreads, 0, s>>>(N.lv[0].D, N.dout, P0,
                                                               N.theta + Hd.woff, N.T1,
                                                               N.grad + Hd.woff);
    else
        netk::k_head_bwd<64><<<gh, netk::kElemThreads, 0, s>>>(N.lv[0].D, N.dout, P0,
                                                               N.theta + Hd.woff, N.T1,
                                                               N.grad + Hd.woff);
    NLH_CHECK_LAUNCH();
    // decoder, finest level first; T1 holds the gradient of D_l (l = 0: from
    // the head, same resolution; l > 0: the upsampled part of dec_{l-1}a's
    // input gradient, one level finer)
    for (int l = 0; l <= Lv - 2; ++l) {
        const int h = H >> l, w = W >> l;
        Level &L = N.lv[l];
        const int lb = N.index(false, l, 1), la = N.index(false, l, 0);
        grad_merge(N, lb, l == 0 ? N.T1 : nullptr, nullptr, l == 0 ? nullptr : N.T1, L.D, B, h, w,
                   s);
        conv_wgrad(N, lb, netk::Src{L.DA, N.ch(l), 0, nullptr, 0}, N.dz, B, h, w, s);
        conv_dgrad(N, lb, N.dz, B, h, w, N.T2, N.ch(l), nullptr, s);
        grad_merge(N, la, N.T2, nullptr, nullptr, L.DA, B, h, w, s);
        const bf16 *coarse = l == Lv - 2 ? N.lv[l + 1].E : N.lv[l + 1].D;
        conv_wgrad(N, la, netk::Src{coarse, N.ch(l + 1), 1, L.E, N.ch(l)}, N.dz, B, h, w, s);
        conv_dgrad(N, la, N.dz, B, h, w, N.T1, N.ch(l + 1), L.S, s);
    }
    // encoder, coarsest level first; at the bottom T1 is the upsample
    // gradient (finer), above it T1 is the pooled-input gradient (coarser)
    for (int l = Lv - 1; l >= 0; --l) {
        const int h = H >> l, w = W >> l;
        Level &L = N.lv[l];
        const int lb = N.index(true, l, 1), la = N.index(true, l, 0);
        if (l == Lv - 1)
            grad_merge(N, lb, nullptr, nullptr, N.T1, L.E, B, h, w, s);
        else
            grad_merge(N, lb, L.S, N.T1, nullptr, L.E, B, h, w, s);
        conv_wgrad(N, lb, netk::Src{L.A, N.ch(l), 0, nullptr, 0}, N.dz, B, h, w, s);
        conv_dgrad(N, lb, N.dz, B, h, w, N.T2, N.ch(l), nullptr, s);
        grad_merge(N, la, N.T2, nullptr, nullptr, L.A, B, h, w, s);
        const bf16 *in = l == 0 ? N.X0 : L.Q;
        const int cin = l == 0 ? 32 : N.ch(l - 1);
        conv_wgrad(N, la, netk::Src{in, cin, 0, nullptr, 0}, N.dz, B, h, w, s);
        if (l > 0) conv_dgrad(N, la, N.dz, B, h, w, N.T1, cin, nullptr, s);
    }
}

static nlh_net_s *checked(nlh_net net) {
    NLH_REQUIRE(net, "net is NULL");
    return net;
}

// After a synchronisation: throw NLH_ERR_TIMEOUT (and clear the word) if a
// tensor-core wait gave up since the last check.
static void take_error(nlh_net_s &N) {
    int e = 0;
    NLH_CUDA(cudaMemcpy(&e, N.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        NLH_CUDA(cudaMemset(N.err, 0, sizeof(int)));
        set_error("net: a bounded tensor-core wait gave up; results of the call are invalid");
        throw Failure{NLH_ERR_TIMEOUT};
    }
}

extern "C" {

nlh_status nlh_net_create(int base, int levels, nlh_net *out) {
    clear_error();
    nlh_net_s *N = nullptr;
    try {
        NLH_REQUIRE(out, "nlh_net_create: out is NULL");
        *out = nullptr;
        NLH_REQUIRE(base == 32 || base == 64, "nlh_net_create: base must be 32 or 64");
        NLH_REQUIRE(levels >= 2 && levels <= 4, "nlh_net_create: levels must be in [2, 4]");
        N = new nlh_net_s();
        N->base = base;
        N->levels = levels;
        auto add = [&](int cin, int cout, int k) {
            LayerDesc d{};
            d.cin = cin, d.cout = cout, d.k = k;
            d.cinp = (cin + 31) / 32 * 32;
            d.woff = N->n_params;
            N->n_params += (int64_t)cout * k * k * cin;
            d.boff = N->n_params;
            N->n_params += cout;
            if (k == 3) {
                d.wfoff = N->wf_total;
                d.wdoff = N->wf_total;
                N->wf_total += (int64_t)cout * 9 * d.cinp;
            }
            N->layers.push_back(d);
        };
        int cin = 3;
        for (int l = 0; l < levels; ++l) {
            add(cin, base << l, 3);
            add(base << l, base << l, 3);
            cin = base << l;
        }
        for (int l = levels - 2; l >= 0; --l) {
            add((base << (l + 1)) + (base << l), base << l, 3);
            add(base << l, base << l, 3);
        }
        add(base, 2, 1);
        netk::PackTable &t = N->pack;
        t.nl = (int)N->layers.size() - 1;
        t.start[0] = 0;
        for (int l = 0; l < t.nl; ++l) {
            const LayerDesc &d = N->layers[l];
            t.cin[l] = d.cin, t.cinp[l] = d.cinp, t.cout[l] = d.cout;
            t.woff[l] = d.woff, t.wfoff[l] = d.wfoff, t.wdoff[l] = d.wdoff;
            t.start[l + 1] = t.start[l] + (int64_t)d.cout * 9 * d.cinp;
        }
        NLH_CUDA(cudaMalloc(&N->theta, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMalloc(&N->grad, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMalloc(&N->m, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMalloc(&N->v, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMalloc(&N->wf, sizeof(bf16) * N->wf_total));
        NLH_CUDA(cudaMalloc(&N->wd, sizeof(bf16) * N->wf_total));
        NLH_CUDA(cudaMalloc(&N->wtf, sizeof(bf16) * N->wf_total));
        NLH_CUDA(cudaMalloc(&N->wtd, sizeof(bf16) * N->wf_total));
        NLH_CUDA(cudaMemset(N->theta, 0, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMemset(N->grad, 0, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMemset(N->m, 0, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMemset(N->v, 0, sizeof(float) * N->n_params));
        NLH_CUDA(cudaMalloc(&N->err, sizeof(int)));
        NLH_CUDA(cudaMemset(N->err, 0, sizeof(int)));
        *out = N;
        return NLH_OK;
    } catch (Failure &f) {
        delete N;
        return f.st;
    }
}

nlh_status nlh_net_info(nlh_net net, int *n_layers, int64_t *n_params) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        if (n_layers) *n_layers = (int)N->layers.size();
        if (n_params) *n_params = N->n_params;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_layer(nlh_net net, int i, int *cin, int *cout, int *k) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(i >= 0 && i < (int)N->layers.size(), "nlh_net_layer: index out of range");
        if (cin) *cin = N->layers[i].cin;
        if (cout) *cout = N->layers[i].cout;
        if (k) *k = N->layers[i].k;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_set_params(nlh_net net, const float *theta, int64_t count) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(theta && count == N->n_params, "nlh_net_set_params: expected %lld floats",
                    (long long)N->n_params);
        NLH_CUDA(cudaDeviceSynchronize());
        NLH_CUDA(cudaMemcpy(N->theta, theta, sizeof(float) * count, cudaMemcpyHostToDevice));
        NLH_CUDA(cudaMemset(N->m, 0, sizeof(float) * count));
        NLH_CUDA(cudaMemset(N->v, 0, sizeof(float) * count));
        N->adam_t = 0;
        N->packed = false;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

static nlh_status copy_out(nlh_net net, bool grads, float *dst, int64_t count) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(dst && count == N->n_params, "nlh_net_get_%s: expected %lld floats",
                    grads ? "grads" : "params", (long long)N->n_params);
        NLH_CUDA(cudaDeviceSynchronize());
        take_error(*N);
        NLH_CUDA(cudaMemcpy(dst, grads ? N->grad : N->theta, sizeof(float) * count,
                            cudaMemcpyDeviceToHost));
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_get_params(nlh_net net, float *theta, int64_t count) {
    return copy_out(net, false, theta, count);
}

nlh_status nlh_net_get_grads(nlh_net net, float *grad, int64_t count) {
    return copy_out(net, true, grad, count);
}

nlh_status nlh_net_forward(nlh_net net, const nlh_net_batch *batch, double *u0, double *scale,
                           void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        check_batch(*N, batch);
        cudaStream_t s = (cudaStream_t)stream;
        net_ensure_ws(*N, batch->B, batch->H, batch->W, false, s);
        net_forward(*N, *batch, u0, scale, nullptr, s);
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_residual_error(nlh_net net, const nlh_net_batch *batch, double *e0,
                                  void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        check_batch(*N, batch);
        NLH_REQUIRE(batch->ustar && e0, "nlh_net_residual_error: ustar and e0 are required");
        cudaStream_t s = (cudaStream_t)stream;
        net_ensure_ws(*N, batch->B, batch->H, batch->W, false, s);
        // u0 goes to e0, then e0 = ustar - u0 in place
        net_forward(*N, *batch, e0, nullptr, nullptr, s);
        const int64_t n = (int64_t)batch->B * batch->H * batch->W;
        netk::k_sub<<<grid_for(n, 256), 256, 0, s>>>(batch->ustar, e0, n, e0);
        NLH_CHECK_LAUNCH();
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_loss_grad(nlh_net net, const nlh_net_batch *batch, double *loss,
                             void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        check_batch(*N, batch);
        const nlh_net_batch &b = *batch;
        NLH_REQUIRE(b.ustar && b.deg, "nlh_net_loss_grad: ustar and deg are required");
        NLH_REQUIRE(b.beta >= 0.0, "nlh_net_loss_grad: beta must be >= 0");
        if (b.beta > 0.0)
            NLH_REQUIRE(b.e0 && b.r0, "nlh_net_loss_grad: beta > 0 needs e0 and r0");
        cudaStream_t s = (cudaStream_t)stream;
        net_ensure_ws(*N, b.B, b.H, b.W, true, s);
        net_forward(*N, b, nullptr, nullptr, b.beta > 0.0 ? b.e0 : nullptr, s);
        const int HW = b.H * b.W;
        const int64_t P0 = (int64_t)b.B * HW;
        NLH_CUDA(cudaMemsetAsync(N->loss, 0, sizeof(double), s));
        netk::k_loss_grad<<<std::min(grid_for(P0, netk::kElemThreads), 2 * kSMs),
                            netk::kElemThreads, 0, s>>>(N->o, b.ustar, b.r0, b.e0, b.deg,
                                                        N->stats, make_scalars(b), b.B, HW,
                                                        b.beta, N->dout, N->loss);
        NLH_CHECK_LAUNCH();
        net_backward(*N, b, s);
        if (loss) {
            NLH_CUDA(cudaMemcpyAsync(loss, N->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
            NLH_CUDA(cudaStreamSynchronize(s));
            take_error(*N);
        }
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_adam(nlh_net net, double lr, double beta1, double beta2, double eps,
                        void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(lr > 0 && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0,
                    "nlh_net_adam: bad hyper-parameters");
        cudaStream_t s = (cudaStream_t)stream;
        N->adam_t += 1;
        const double c1 = 1.0 / (1.0 - std::pow(beta1, N->adam_t));
        const double c2 = 1.0 / (1.0 - std::pow(beta2, N->adam_t));
        netk::k_adam<<<grid_for(N->n_params, 256), 256, 0, s>>>(
            N->theta, N->grad, N->m, N->v, N->n_params, (float)lr, (float)beta1,
            (float)(1.0 - beta1), (float)beta2, (float)(1.0 - beta2), (float)eps, (float)c1,
            (float)c2);
        NLH_CHECK_LAUNCH();
        N->packed = false;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_set_engine(nlh_net net, int engine) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(engine == NLH_NET_ENGINE_MMA_SYNC || engine == NLH_NET_ENGINE_TCGEN05,
                    "nlh_net_set_engine: engine must be 0 (mma.sync) or 1 (tcgen05)");
        N->engine = engine;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_get_engine(nlh_net net, int *engine) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_REQUIRE(engine, "nlh_net_get_engine: engine is NULL");
        *engine = N->engine;
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_check(nlh_net net, void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        NLH_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        take_error(*N);
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_selftest_net_timeout(nlh_net net, void *stream) {
    clear_error();
    try {
        nlh_net_s *N = checked(net);
        k_selftest_wait_nothing<<<1, 32, 0, (cudaStream_t)stream>>>(N->err);
        NLH_CHECK_LAUNCH();
        return NLH_OK;
    } catch (Failure &f) {
        return f.st;
    }
}

nlh_status nlh_net_destroy(nlh_net net) {
    clear_error();
    delete net;
    return NLH_OK;
}

}  // extern "C"
