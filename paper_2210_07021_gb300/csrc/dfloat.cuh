// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two FP32 numbers; after
// normalisation |l| <= ulp(h)/2, which carries about 48 significant bits.
// The building blocks are the error-free transformations of a sum
// (Knuth, TAOCP vol. 2, Sec. 4.2.2: two-sum; Dekker 1971: fast two-sum when
// |a| >= |b|) and of a product (the fused multiply-add returns the rounding
// error of a*b exactly).  On this GPU the FP32 pipe issues 64 times as many
// fused multiply-adds per clock as the FP64 pipe, so a double-float operation
// of 4 to 11 FP32 instructions is several times faster than its FP64 twin
// while keeping the 1e-10 accuracy target within reach.
//
// Every operation uses explicitly rounded intrinsics (__fadd_rn and so on),
// which the compiler neither contracts nor reorders, so the error-free
// transformations stay exact whatever -fmad setting the file is built with.
#pragma once

#include <cuda_runtime.h>

namespace sfmm {

struct __align__(8) dflt {
    float h, l;
    dflt() = default;
    __host__ __device__ constexpr dflt(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ dflt(int v) : h((float)v), l(0.f) {}            // exact for |v| < 2^24
    __host__ __device__ dflt(float v) : h(v), l(0.f) {}
    // rounding of an FP64 value: h = fl32(v), l = fl32(v - h)
    __host__ __device__ explicit dflt(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ dflt dfl_fast_two_sum(float a, float b)     // requires |a| >= |b| (or a == 0)
{
    const float s = __fadd_rn(a, b);
    return dflt(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dflt dfl_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dflt(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dflt dfl_norm(dflt a) { return dfl_fast_two_sum(a.h, a.l); }

__device__ __forceinline__ dflt operator+(dflt a, dflt b)
{
    const dflt s = dfl_two_sum(a.h, b.h);
    return dfl_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dflt operator-(dflt a) { return dflt(-a.h, -a.l); }
__device__ __forceinline__ dflt operator-(dflt a, dflt b) { return a + (-b); }
__device__ __forceinline__ dflt operator*(dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);
    return dfl_fast_two_sum(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}
__device__ __forceinline__ dflt operator*(dflt a, float b)
{
    const float p = __fmul_rn(a.h, b);
    const float e = __fmaf_rn(a.h, b, -p);
    return dfl_fast_two_sum(p, __fmaf_rn(a.l, b, e));
}
// a / b: quotient of the leading parts, one correction from the remainder
__device__ __forceinline__ dflt operator/(dflt a, dflt b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const dflt r = a - b * q1;
    const float q2 = __fdiv_rn(r.h, b.h);
    return dfl_fast_two_sum(q1, q2);
}
__device__ __forceinline__ dflt& operator+=(dflt& a, dflt b) { a = a + b; return a; }
__device__ __forceinline__ dflt& operator*=(dflt& a, dflt b) { a = a * b; return a; }

// Product left unnormalised (|l| may exceed ulp(h)/2): for operands that feed
// dfl_mac straight away.
__device__ __forceinline__ dflt dfl_mul_lazy(dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    return dflt(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p))));
}
// acc += a * b without renormalising acc: the leading parts meet in an exact
// two-sum, every error term is added to acc.l.  Over n terms acc.l grows like
// n ulp(acc.h), so its own rounding stays near n 2^-48 |acc|; call dfl_norm
// once at the end.
__device__ __forceinline__ void dfl_mac(dflt& acc, dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
    const dflt s = dfl_two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}

// log x for a double-float x > 0 (normal leading part), left unnormalised for
// an accumulation.  tab[j] (j < 128) holds log c_j and 1/c_j as (hi, lo) pairs,
// tab[128] log 2 as a 16-bit leading part and the rest; the tables are rounded
// from FP64 on the host.  x = 2^e m (1 + l'), m in [1, 2); with c_j = 1 + j/128 the
// leading seven fraction bits of m, log x = e log 2 + log c_j + log1p(r),
// r = (m - c_j + l 2^-e) / c_j, |r| < 2^-7.  m - c_j is exact; log1p(r) - r is
// a degree-6 series (remainder below r^7/7 < 2^-52); log 2 is split so that
// e times its leading part is exact.  The three leading terms meet in two
// exact two-sums, every tail goes to the low part.
__device__ __forceinline__ dflt dfl_log_lazy(dflt x, const float4* __restrict__ tab)
{
    const int bits = __float_as_int(x.h);
    const int be = bits >> 23;                                            // biased exponent (x.h > 0)
    const int j = (bits >> 16) & 0x7F;
    const float m = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);     // [1, 2)
    const float cj = __int_as_float((bits & 0x007F0000) | 0x3F800000);    // 1 + j/128, exactly
    const float scale = __int_as_float((254 - be) << 23);                 // 2^-e
    const float4 t = tab[j];                                              // log c_j (hi, lo), 1/c_j (hi, lo)
    const dflt delta = dfl_two_sum(__fsub_rn(m, cj), __fmul_rn(x.l, scale));
    const dflt r = dfl_mul_lazy(delta, dflt(t.z, t.w));
    const float rh = r.h;
    float poly = __fmul_rn(rh, rh) * (-0.5f + rh * (1.f / 3.f + rh * (-0.25f + rh * (0.2f + rh * (-1.f / 6.f)))));
    poly = __fmaf_rn(-rh, r.l, poly);                                     // cross term of -r^2/2
    const float4 l2 = tab[128];                                           // log 2: 16-bit leading part, tail
    const float e = (float)(be - 127);
    const dflt s1 = dfl_two_sum(__fmul_rn(e, l2.x), t.x);
    const dflt s2 = dfl_two_sum(s1.h, rh);
    const float lo = __fmaf_rn(e, l2.y, __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(t.y, r.l), poly)));
    return dflt(s2.h, lo);
}

__device__ __forceinline__ dflt dfl_shfl_up(dflt v, int o)
{
    return dflt(__shfl_up_sync(0xffffffffu, v.h, o), __shfl_up_sync(0xffffffffu, v.l, o));
}
__device__ __forceinline__ dflt dfl_shfl_xor(dflt v, int o)
{
    return dflt(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

}  // namespace sfmm
