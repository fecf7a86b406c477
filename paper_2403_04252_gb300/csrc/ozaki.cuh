// Error-free building blocks of the FP64-accurate tensor-core contraction (precision modes 4 and 5).
//
// Values are carried as unevaluated sums of two floats ("double-float", hi + lo with |lo| <= ulp(hi)),
// about 48 significant bits, so that the per-node products run on the FP32 pipe instead of the
// much narrower FP64 pipe.  For the tensor cores, each value of a 128-node window (four 32-node
// chunks) is written in fixed point against a power-of-two scale s chosen from the largest |value| of
// its row in the window,
//   x = s sum_{i < OZ_SLICES} k_i 2^(-8 i),   k_i integers with |k_i| <= 129,
// and slice i is stored as the bf16 number k_i 2^(-8 i), which is exact (k_i has at most 8 significant
// bits).  This is the error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) with a fixed-point
// grid per window.  Seven slices keep 55 bits below the window maximum; the products of two sliced
// values with i + j = L <= 3 (at most four per level) are integers times 2^(-8 L) whose sums over 128
// nodes stay below 4 x 128 x 129^2 < 2^24 units, so the tensor core's FP32 accumulator holds each of
// those levels exactly; levels 4 to 6 share one rounded accumulator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace wpccc {

constexpr int OZ_SLICES = 7;   // slices of the FP64-accurate form (the most any layout holds)
constexpr int OZ_FAST_SLICES = 4;   // slices of the reduced-precision tensor-core form (precision mode 3)

// hi + lo = x to about 2^-48 relative (hi = x rounded to FP32, lo = the rest rounded to FP32).
static __device__ __forceinline__ float2 df_split(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return make_float2(h, l);
}

// a b for double-floats a, b: the exact product of the high parts (FMA residual) plus the cross
// terms, renormalised (Fast2Sum: the product's high part dominates).  Relative error ~2^-46.
static __device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float s = p + e;
    return make_float2(s, e - (s - p));
}

// s + err = a + b exactly (Knuth's TwoSum, no ordering assumption).
static __device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// Scale exponent of a chunk row whose largest |value| is mx: the row is multiplied by 2^sh so that its
// largest value lies below 128 (sh = 0 for an all-zero row).  The scale s of the representation is 2^-sh.
static __device__ __forceinline__ int oz_shift(float mx) {
    int E = 0;
    if (mx > 0.f) frexpf(mx, &E);   // mx = f 2^E, f in [0.5, 1)
    return mx > 0.f ? 7 - E : 0;
}

// The first NS bf16 slices k_i 2^(-8 i) of the double-float x = (h, l) scaled by 2^sh (|x| 2^sh < 128).
// The pair (p, e) always holds the remaining value exactly: the scalings by 256 are exact, and so is
// p - k (k is an integer within one of p + e; while p has fraction bits it is below 2^8 in magnitude,
// afterwards p and k are integers below 2^24).  Only p + e may round, which can move k by one where
// the remainder is near a half unit; the next remainder then stays within (0.5 + 2^-17) 256 of zero,
// so |k_i| <= 129.
// NS slices: 7 for FP64 accuracy, 4 for the reduced-precision form (about 31 bits below the window's largest
// value).
template <int NS>
static __device__ __forceinline__ void oz_slices(float h, float l, int sh, __nv_bfloat16 out[NS]) {
    // scaling by 2^sh: one multiplication by the power of two where it is a normal float (as exact as
    // ldexpf: a product with a power of two rounds only where it underflows, and both round the same way)
    float p, e, w = 1.f;
    if (sh >= -126 && sh <= 127) {
        const float s2 = __int_as_float((sh + 127) << 23);
        p = h * s2;
        e = l * s2;
    } else {
        p = ldexpf(h, sh);
        e = ldexpf(l, sh);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const float k = rintf(__fadd_rn(p, e));
        p = __fsub_rn(p, k);
        out[i] = __float2bfloat16_rn(k * w);
        p *= 256.f;
        e *= 256.f;
        w *= (1.f / 256.f);
    }
}

}  // namespace wpccc
