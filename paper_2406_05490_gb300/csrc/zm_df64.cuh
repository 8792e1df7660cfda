// zm_df64.cuh -- double-word arithmetic on pairs of FP32 numbers ("double-float").
//
// A value is x = hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits (unit roundoff
// u^2 = 2^-48 ~ 3.6e-15) in the FP32 exponent range.  GB300 runs FP32 FMA at ~75x its FP64
// rate, so a double-word operation of 6-20 FP32 instructions is several times cheaper than
// one FP64 instruction; the low-order path (stencils, FFT Riesz velocity, RK3 combine) uses
// this arithmetic to stay within FP64-class tolerances without the FP64 pipe.
//
// Building blocks (published error-free transformations, restated here):
//   two_sum       Knuth's TwoSum: s + e == a + b exactly, 6 flops, no precondition;
//   fast_two_sum  Dekker's Fast2Sum: exact when |a| >= |b| (or a == 0), 3 flops;
//   two_prod      p + e == a * b exactly with one FMA (e = fma(a, b, -p)), 2 flops;
// and the double-word algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017):
//   add    "sloppy" sum: error <= c u^2 (|x| + |y|), 11 flops -- normwise accurate, which is
//          what FFT butterflies and sums of like-signed terms need;
//   add_acc accurate sum: relative error <= 3 u^2 even under cancellation, 20 flops;
//   mul    product without the lo*lo term: relative error <= 5 u^2, 8 flops;
//   mul_f  product by an FP32 number: relative error <= 2 u^2, 6 flops.
// Every operation uses the _rn intrinsics, which the compiler never contracts into FMAs or
// reassociates, so the error-free transformations stay exact.
#pragma once

#include <cuda_runtime.h>

namespace zm {
namespace dw {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df mk(float hi, float lo) { return df{hi, lo}; }
__device__ __forceinline__ df from_f(float a) { return df{a, 0.0f}; }
__device__ __forceinline__ df from_f2(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ float2 to_f2(df a) { return make_float2(a.hi, a.lo); }

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ df sub(df x, df y) { return add(x, neg(y)); }

__device__ __forceinline__ df add_acc(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df sub_acc(df x, df y) { return add_acc(x, neg(y)); }

__device__ __forceinline__ df mul(df x, df y)
{
    const df p = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

__device__ __forceinline__ df mul_f(df x, float b)
{
    const df p = two_prod(x.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

__device__ __forceinline__ df sqr(df x)
{
    const df p = two_prod(x.hi, x.hi);
    return fast_two_sum(p.hi, __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, p.lo));
}

// Multiplication by a power of two: exact (barring under/overflow).
__device__ __forceinline__ df scale2(df x, float pow2) { return df{__fmul_rn(x.hi, pow2), __fmul_rn(x.lo, pow2)}; }

// 1 / sqrt(x) for x > 0.  y0 = FP32 estimate (relative error e0 ~ 2^-22).  The residual
// r = 1 - x y0^2 is formed in double-word arithmetic (y0^2 exact by two_prod, 1 - t.hi exact by
// Sterbenz's lemma) and the binomial series y = y0 (1 + r/2 + 3 r^2/8) is applied with the
// leading product y0 r exact, so the result carries the truncation O(e0^3) ~ 2^-66 and a few
// u^2 of rounding (an FP32-rounding emulation measured <= 1.6 u^2 over [0.01, 100]).
__device__ __forceinline__ df rsqrt(df x)
{
    const float y0 = rsqrtf(x.hi);
    const df t = mul(x, two_prod(y0, y0));
    const df r = two_sum(__fsub_rn(1.0f, t.hi), -t.lo);
    const df c = two_prod(y0, r.hi);  // y0 r.hi, exact
    const float rest = __fmaf_rn(y0, r.lo, __fmul_rn(__fmul_rn(c.hi, 0.75f), r.hi));
    const df s = fast_two_sum(y0, __fmul_rn(0.5f, c.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fmul_rn(0.5f, __fadd_rn(c.lo, rest))));
}

// Fused forms for the stencil pass, each one renormalisation instead of several: the rounding
// errors of the leading-part operations are captured exactly (TwoSum / FMA product error) and
// added, with the low parts, in FP32, as in the sloppy sum (normwise error a few u^2).
//   stencil_s:  (m2 - p2) + 8 (p1 - m1)                 28 flops (35 as separate sums)
//   mul_sub:    a b - c d                               19 flops (27)
//   sum_sq3:    x^2 + y^2 + z^2                         31 flops (43), no cancellation
__device__ __forceinline__ df stencil_s(df m2, df m1, df p1, df p2)
{
    const df a = two_sum(m2.hi, -p2.hi);
    const df b = two_sum(p1.hi, -m1.hi);
    const df s = two_sum(a.hi, __fmul_rn(8.0f, b.hi));  // 8 b.hi is exact
    float t = __fadd_rn(__fsub_rn(m2.lo, p2.lo), __fmul_rn(8.0f, __fsub_rn(p1.lo, m1.lo)));
    t = __fadd_rn(t, __fadd_rn(a.lo, __fmaf_rn(8.0f, b.lo, s.lo)));
    return fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df mul_sub(df a, df b, df c, df d)
{
    const df p = two_prod(a.hi, b.hi);
    const df q = two_prod(c.hi, d.hi);
    const df s = two_sum(p.hi, -q.hi);
    float t = __fadd_rn(s.lo, __fsub_rn(p.lo, q.lo));
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    t = __fmaf_rn(-c.hi, d.lo, t);
    t = __fmaf_rn(-c.lo, d.hi, t);
    return fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df sum_sq3(df x, df y, df z)
{
    const df a = two_prod(x.hi, x.hi), b = two_prod(y.hi, y.hi), c = two_prod(z.hi, z.hi);
    const df s1 = two_sum(a.hi, b.hi);
    const df s2 = two_sum(s1.hi, c.hi);
    float t = __fadd_rn(__fadd_rn(a.lo, b.lo), c.lo);
    t = __fadd_rn(t, __fadd_rn(s1.lo, s2.lo));
    t = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, t);
    t = __fmaf_rn(__fadd_rn(y.hi, y.hi), y.lo, t);
    t = __fmaf_rn(__fadd_rn(z.hi, z.hi), z.lo, t);
    return fast_two_sum(s2.hi, t);
}

// Complex double-word number, stored as float4 {re.hi, re.lo, im.hi, im.lo}.
struct cdf {
    df re, im;
};

__device__ __forceinline__ cdf ld_c(float4 v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ __forceinline__ float4 st_c(cdf a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{sub(a.re, b.re), sub(a.im, b.im)}; }
__device__ __forceinline__ cdf cmul(cdf a, cdf b)
{
    return cdf{sub(mul(a.re, b.re), mul(a.im, b.im)), add(mul(a.re, b.im), mul(a.im, b.re))};
}
// a * (+i) when s > 0, a * (-i) when s < 0: exact (a swap and a sign).
__device__ __forceinline__ cdf cmul_pm_i(cdf a, int s)
{
    return s > 0 ? cdf{neg(a.im), a.re} : cdf{a.im, neg(a.re)};
}

// ---- complex double words in packed FP32x2 instructions ------------------------------------
// One complex double word as two 64-bit registers: h = (re.hi, im.hi), l = (re.lo, im.lo); each
// fma/mul/add/sub .f32x2 instruction applies the same FP32 operation to both lanes, so the real
// and imaginary parts of an operation share one issue slot.  In memory: {re.hi, im.hi, re.lo,
// im.lo} (16 bytes, read and written as ulonglong2).
using u64 = unsigned long long;

__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
constexpr u64 kSign0 = 0x0000000080000000ull, kSign1 = 0x8000000000000000ull;
__device__ __forceinline__ u64 neg2(u64 a) { return a ^ (kSign0 | kSign1); }
__device__ __forceinline__ u64 pk(float x, float y)
{
    return (u64)__float_as_uint(x) | ((u64)__float_as_uint(y) << 32);
}
__device__ __forceinline__ float lane0(u64 a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float lane1(u64 a) { return __uint_as_float((unsigned)(a >> 32)); }
// (x, y) -> (-y, x)
__device__ __forceinline__ u64 rot2(u64 a) { return pk(-lane1(a), lane0(a)); }

struct C2 {
    u64 h, l;
};

__device__ __forceinline__ C2 ld2(ulonglong2 v) { return C2{v.x, v.y}; }
__device__ __forceinline__ ulonglong2 st2(C2 a) { return make_ulonglong2(a.h, a.l); }
__device__ __forceinline__ C2 c2_from(df re, df im) { return C2{pk(re.hi, im.hi), pk(re.lo, im.lo)}; }
__device__ __forceinline__ df c2_re(C2 a) { return df{lane0(a.h), lane0(a.l)}; }

__device__ __forceinline__ void two_sum2(u64 a, u64 b, u64 &s, u64 &e)
{
    s = add2(a, b);
    const u64 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// s + e == a - b exactly (two_sum of a and -b)
__device__ __forceinline__ void two_diff2(u64 a, u64 b, u64 &s, u64 &e)
{
    s = sub2(a, b);
    const u64 bb = sub2(s, a);
    e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
__device__ __forceinline__ C2 fast_two_sum2(u64 a, u64 b)
{
    const u64 s = add2(a, b);
    return C2{s, sub2(b, sub2(s, a))};
}

// sloppy double-word sums of both parts (11 packed instructions)
__device__ __forceinline__ C2 cadd2(C2 x, C2 y)
{
    u64 s, e;
    two_sum2(x.h, y.h, s, e);
    return fast_two_sum2(s, add2(e, add2(x.l, y.l)));
}
__device__ __forceinline__ C2 csub2(C2 x, C2 y)
{
    u64 s, e;
    two_diff2(x.h, y.h, s, e);
    return fast_two_sum2(s, add2(e, sub2(x.l, y.l)));
}

// The same sums without the final renormalisation (8 packed instructions): the result
// h + l is exact up to the rounding of the low parts, but |l| may exceed half an ulp of h.  Used
// where the next operation is a sum or product that renormalises (the first layer of a radix-2^2
// butterfly), so the relaxation does not build up.
__device__ __forceinline__ C2 cadd2_lazy(C2 x, C2 y)
{
    u64 s, e;
    two_sum2(x.h, y.h, s, e);
    return C2{s, add2(e, add2(x.l, y.l))};
}
__device__ __forceinline__ C2 csub2_lazy(C2 x, C2 y)
{
    u64 s, e;
    two_diff2(x.h, y.h, s, e);
    return C2{s, add2(e, sub2(x.l, y.l))};
}

// a * w = a wr + (-a.im, a.re) wi, both products exact in their leading parts (two_prod), summed
// with one TwoSum and one renormalisation (19 packed instructions): normwise error a few u^2.
__device__ __forceinline__ C2 cmul2(C2 a, C2 w)
{
    const u64 wrh = pk(lane0(w.h), lane0(w.h)), wrl = pk(lane0(w.l), lane0(w.l));
    const u64 wih = pk(lane1(w.h), lane1(w.h)), wil = pk(lane1(w.l), lane1(w.l));
    const u64 bh = rot2(a.h), bl = rot2(a.l);
    const u64 p1 = mul2(a.h, wrh), p2 = mul2(bh, wih);
    const u64 e1 = fma2(a.h, wrh, neg2(p1)), e2 = fma2(bh, wih, neg2(p2));
    u64 s, e3;
    two_sum2(p1, p2, s, e3);
    u64 t = add2(e1, add2(e2, e3));
    t = fma2(a.l, wrh, t);
    t = fma2(a.h, wrl, t);
    t = fma2(bl, wih, t);
    t = fma2(bh, wil, t);
    return fast_two_sum2(s, t);
}

// a * (+i) for s > 0, a * (-i) for s < 0 (exact)
__device__ __forceinline__ C2 cmul_i2(C2 a, int s)
{
    return s > 0 ? C2{rot2(a.h), rot2(a.l)} : C2{neg2(rot2(a.h)), neg2(rot2(a.l))};
}

}  // namespace dw
}  // namespace zm
