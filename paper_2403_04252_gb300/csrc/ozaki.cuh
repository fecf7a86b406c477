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
// nodes stay below 4 x 128 x 130^2 < 2^24 units, so the tensor core's FP32 accumulator holds each of
// those levels exactly; levels 4 to 6 share one rounded accumulator.  (The four-slice generated operand
// of the reduced-precision form is sliced by grid rounding, oz_slices4_pe_x2, with |k_i| <= 130.)
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

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

// Two bf16 numbers held exactly in floats (low 16 bits zero) packed as bf16x2: lo in the low half.
static __device__ __forceinline__ uint32_t bf16x2_exact(float lo, float hi) {
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Pairs of floats in one 64-bit register, operated on by the packed FP32x2 instructions (one
// instruction per pair, each half rounded as its own IEEE operation).
struct f32x2 {
    uint64_t v;
};
static __device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
static __device__ __forceinline__ void x2_unpack(f32x2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
static __device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
static __device__ __forceinline__ f32x2 x2_neg(f32x2 a) { return f32x2{a.v ^ 0x8000000080000000ull}; }

// w a for double-floats w, a at two nodes at once ((wh, wl) and (ah, al) hold the two nodes' high and low
// parts) as unnormalised pairs p + e: p = fl(wh ah), e = its FMA residual plus the cross terms, so
// |e| <= 3 2^-24 |p| (to first order) and p + e carries w a to about 2^-46 relative.
static __device__ __forceinline__ void df_mul_pe_x2(f32x2 wh, f32x2 wl, f32x2 ah, f32x2 al, f32x2& p, f32x2& e) {
    p = x2_mul(wh, ah);
    e = x2_fma(wh, ah, x2_neg(p));
    e = x2_fma(wh, al, e);
    e = x2_fma(wl, ah, e);
}

// The four fixed-point slices of the pairs p + e of two nodes scaled by s2 = 2^sh in both halves
// (|p s| < 128, |e| <= 2^-21 |p|), each rounded to its grid by adding and subtracting 1.5 2^23 times the
// grid unit (1, 2^-8, 2^-16, 2^-24):
//   t0 = RN(p s),  t1 = RN_{2^-8}(p s - t0),  t2 = RN_{2^-16}(p s - t0 - t1 + e s),  t3 = RN_{2^-24}(rest).
// Every remainder is exact (a multiple of its operand's unit, smaller than it) except the one that
// brings in e s, which rounds by at most 2^-33; so |p s + e s - sum t_i| <= 2^-25 + 2^-33, and every t_i is
// k_i 2^(-8 i) with |k_i| <= 130 (a bf16 number: its low 16 bits are zero), as the tensor-core levels need.
static __device__ __forceinline__ void oz_slices4_pe_x2(f32x2 p, f32x2 e, f32x2 s2, f32x2 t[4]) {
    const f32x2 C0 = x2_pack(12582912.f, 12582912.f), C1 = x2_pack(49152.f, 49152.f),
                C2 = x2_pack(192.f, 192.f), C3 = x2_pack(0.75f, 0.75f);
    const f32x2 P = x2_mul(p, s2);   // exact: a power-of-two scaling of a value below 128 times the scale
    t[0] = x2_sub(x2_add(P, C0), C0);
    const f32x2 r0 = x2_sub(P, t[0]);
    t[1] = x2_sub(x2_add(r0, C1), C1);
    const f32x2 r1 = x2_sub(r0, t[1]);
    const f32x2 s1 = x2_fma(e, s2, r1);
    t[2] = x2_sub(x2_add(s1, C2), C2);
    const f32x2 r2 = x2_sub(s1, t[2]);
    t[3] = x2_sub(x2_add(r2, C3), C3);
}

// s + err = a + b exactly on two pairs at once (TwoSum).
static __device__ __forceinline__ f32x2 two_sum_x2(f32x2 a, f32x2 b, f32x2& err) {
    const f32x2 s = x2_add(a, b);
    const f32x2 bb = x2_sub(s, a);
    err = x2_add(x2_sub(a, x2_sub(s, bb)), x2_sub(b, bb));
    return s;
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
