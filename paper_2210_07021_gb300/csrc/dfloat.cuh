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

// The float m 2^e for an integer 2^23 <= m < 2^24, built from its bits; zero
// (with the sign) below the normal range.
__device__ __forceinline__ float dfl_float_m24(uint32_t m, int e, uint32_t sign)
{
    const int be = e + 23 + 127;
    if (m == 0u || be <= 0) return __uint_as_float(sign);
    return __uint_as_float(sign | ((uint32_t)be << 23) | (m & 0x7FFFFFu));
}

// a - b for FP64 a, b as a normalised double-float, with integer and FP32
// instructions only (this GPU's FP64 pipe issues 1/64 of the FP32 rate, so
// bulk conversions of FP64 data are faster this way).  The mantissas are
// brought to the larger exponent lowered by up to 9 bits; their difference is
// then exact in a 64-bit integer unless the exponents differ by more than 9,
// when the smaller operand is below 2^-9 of the larger and the bits shifted
// out lie under 2^-61 of the result.  The leading 24 bits of the difference
// give hi, the next 24 lo, and a fast two-sum rounds the pair to normal form:
// hi + lo equals a - b to 2^-47 relative (exactly when it has <= 48 bits, e.g.
// a point and a box centre 2^-5 apart on the unit sphere), up to an absolute
// 2^-126: parts below the normal range are flushed to zero.
__device__ __forceinline__ dflt dfl_sub_exact(double a, double b)
{
    const long long ua = __double_as_longlong(a), ub = __double_as_longlong(b);
    int ea = (int)((ua >> 52) & 0x7FF), eb = (int)((ub >> 52) & 0x7FF);
    long long ma = ua & 0x000FFFFFFFFFFFFFLL, mb = ub & 0x000FFFFFFFFFFFFFLL;
    if (ea) ma |= 1LL << 52; else ea = 1;            // subnormal: exponent 1, no leading bit
    if (eb) mb |= 1LL << 52; else eb = 1;
    if (ua < 0) ma = -ma;
    if (ub < 0) mb = -mb;
    const bool swap = eb > ea;                       // make ea >= eb; the difference changes sign
    if (swap) {
        const int te = ea; ea = eb; eb = te;
        const long long tm = ma; ma = mb; mb = tm;
    }
    const int k = min(9, ea - eb);
    const int r = ea - eb - k;
    const long long d0 = ma * (1LL << k) - (r < 63 ? (mb >> r) : 0LL);   // |d0| < 2^62 + 2^53
    if (d0 == 0) return dflt(0.f, 0.f);
    const long long d = swap ? -d0 : d0;             // a - b = d 2^(ea - k - 1075)
    const uint32_t sign = d < 0 ? 0x80000000u : 0u;
    unsigned long long u = (unsigned long long)(d < 0 ? -d : d);
    const int lz = __clzll((long long)u);
    u <<= lz;                                        // leading bit at 2^63: a - b = u 2^(e0 - lz)
    const int e0 = ea - k - 1075;
    const float hi = dfl_float_m24((uint32_t)(u >> 40), e0 - lz + 40, sign);
    const unsigned long long rest = u & ((1ULL << 40) - 1ULL);
    float lo = 0.f;
    if (rest != 0ULL) {
        const int lz2 = __clzll((long long)rest);
        lo = dfl_float_m24((uint32_t)((rest << lz2) >> 40), e0 - lz - lz2 + 40, sign);
    }
    return dfl_fast_two_sum(hi, lo);
}

// sqrt of a double-float x >= 0: the FP32 root and one correction from the exact remainder
__device__ __forceinline__ dflt dfl_sqrt(dflt x)
{
    if (!(x.h > 0.f)) return dflt(0.f, 0.f);
    const float s = sqrtf(x.h);
    const float r = __fadd_rn(__fmaf_rn(-s, s, x.h), x.l);
    return dfl_fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

// 1/k as double-float pairs, k = 1..12 (rounded from FP64 at compile time)
struct InvTabDF {
    float h[13], l[13];
};
constexpr InvTabDF make_inv_tab()
{
    InvTabDF t{};
    for (int k = 1; k <= 12; ++k) {
        const double v = 1.0 / k;
        t.h[k] = (float)v;
        t.l[k] = (float)(v - (double)(float)v);
    }
    return t;
}
namespace {
__constant__ InvTabDF kInvDF = make_inv_tab();
}  // namespace

// log(1 - x) for a double-float 0 <= x < 1, to double-float accuracy relative
// to the result: below x = 2^-5 the series -x (1 + x/2 + ... + x^11/12)
// (remainder under x^13/13 < 2^-64 x), else the table logarithm of 1 - x
// (whose absolute error 2^-48 is then below 2^-43 of the result).
__device__ __forceinline__ dflt dfl_log1m(dflt x, const float4* tab)
{
    if (x.h < 0.03125f) {
        dflt acc(kInvDF.h[12], kInvDF.l[12]);
        for (int k = 11; k >= 1; --k) acc = dflt(kInvDF.h[k], kInvDF.l[k]) + x * acc;
        return -(x * acc);
    }
    return dfl_norm(dfl_log_lazy(dflt(1.f, 0.f) - x, tab));
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
