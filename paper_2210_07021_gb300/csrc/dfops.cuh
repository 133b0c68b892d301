// Double-float building blocks of the thread-per-translation kernels
// (m2l_pair.cu, updown_df.cu): lazy sums and products, complex products,
// and the two binomial passes of the translations of Lemmas 2-4 in place on a
// register array.
#pragma once
#include "dfloat.cuh"

namespace sfmm {

// a + b with the low parts summed but not renormalised (an exact two-sum of the
// leading parts; its error and both tails go to the low part)
__device__ __forceinline__ dflt add_lazy(dflt a, dflt b)
{
    const dflt s = dfl_two_sum(a.h, b.h);
    return dflt(s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l));
}
// renormalisation safe for any magnitudes of the two parts
__device__ __forceinline__ dflt renorm(dflt a) { return dfl_two_sum(a.h, a.l); }

// (ar + i ai)(br + i bi): per part, the two leading products meet in one exact
// two-sum and every rounding error goes to the low part
__device__ __forceinline__ void cmul_df(dflt ar, dflt ai, dflt br, dflt bi, dflt* cr, dflt* ci)
{
    const float p1 = __fmul_rn(ar.h, br.h), p2 = __fmul_rn(ai.h, bi.h);
    const float p3 = __fmul_rn(ar.h, bi.h), p4 = __fmul_rn(ai.h, br.h);
    const float e1 = __fmaf_rn(ar.h, br.l, __fmaf_rn(ar.l, br.h, __fmaf_rn(ar.h, br.h, -p1)));
    const float e2 = __fmaf_rn(ai.h, bi.l, __fmaf_rn(ai.l, bi.h, __fmaf_rn(ai.h, bi.h, -p2)));
    const float e3 = __fmaf_rn(ar.h, bi.l, __fmaf_rn(ar.l, bi.h, __fmaf_rn(ar.h, bi.h, -p3)));
    const float e4 = __fmaf_rn(ai.h, br.l, __fmaf_rn(ai.l, br.h, __fmaf_rn(ai.h, br.h, -p4)));
    const dflt s = dfl_two_sum(p1, -p2), t = dfl_two_sum(p3, p4);
    *cr = dfl_fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(e1, e2)));
    *ci = dfl_fast_two_sum(t.h, __fadd_rn(t.l, __fadd_rn(e3, e4)));
}

// The Taylor shift by one in place: for i < P, for j = P-1 down to i,
// c_j += c_{j+1} (c_n = sum_{l >= n} C(l, n) c_l).  The passes run in groups
// of four: a group's body is unrolled over j >= its first pass (so c stays in
// registers) and its passes are a runtime loop, with the j < i positions
// left alone: about a quarter of the code of fully unrolled passes (which
// overflows the instruction cache at P = 20), for about 15 % more additions.
template <int P>
__device__ __forceinline__ void pascal_up(dflt* c)
{
#pragma unroll
    for (int g = 0; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j] = add_lazy(c[j], c[j + 1]);
        }
    }
}

// Its dual on x_m = c[m + 1], m = 0..P-1: for i = 1..P-1, for j = P-1 down to i,
// x_j += x_{j-1} (x_k = sum_{m <= k} C(k, m) x_m), grouped the same way.
template <int P>
__device__ __forceinline__ void pascal_down(dflt* c)
{
#pragma unroll
    for (int g = 1; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4 && i < P; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j + 1] = add_lazy(c[j + 1], c[j]);
        }
    }
}

__device__ __forceinline__ dflt ld_dflt2(const dflt* p, dflt* second)
{
    const float4 v = *reinterpret_cast<const float4*>(p);   // 16-byte aligned (Re, Im) pair
    *second = dflt(v.z, v.w);
    return dflt(v.x, v.y);
}

// acc + a b with the low part unnormalised: the leading parts meet in an exact
// two-sum, the product's rounding error and the tails go to the low part
__device__ __forceinline__ dflt mac_lazy(dflt acc, dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
    const dflt s = dfl_two_sum(acc.h, p);
    return dflt(s.h, __fadd_rn(acc.l, __fadd_rn(s.l, e)));
}

// The Taylor shift by a: for i < P, for j = P-1 down to i, c_j += a c_{j+1}
// (c_n = sum_{l >= n} C(l, n) a^(l-n) c_l), grouped as pascal_up.
template <int P>
__device__ __forceinline__ void pascal_up_mul(dflt* c, dflt a)
{
#pragma unroll
    for (int g = 0; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j] = mac_lazy(c[j], a, c[j + 1]);
        }
    }
}

// Its dual with multiplier b on x_m = c[m + 1]: for i = 1..P-1, for j = P-1
// down to i, x_j += b x_{j-1} (x_k = sum_{m <= k} C(k, m) b^(k-m) x_m).
template <int P>
__device__ __forceinline__ void pascal_down_mul(dflt* c, dflt b)
{
#pragma unroll
    for (int g = 1; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4 && i < P; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j + 1] = mac_lazy(c[j + 1], b, c[j]);
        }
    }
}

// ------------------------------------------------------------------------
// Packed pairs: the real and imaginary parts of a coefficient as one
// double-float pair of float2, so that each FP32x2 instruction does the work
// of two (the binomial passes treat both parts alike).  x - y is taken as
// fma(y, -1, x), exact in its product, so the error-free transformations keep
// their exactness.
struct dflt2 {
    float2 h, l;
};

__device__ __forceinline__ float2 f2s(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2s(-1.f), x); }

__device__ __forceinline__ dflt2 two_sum2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    const float2 e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
    return dflt2{s, e};
}
__device__ __forceinline__ dflt2 fast_two_sum2(float2 a, float2 b)     // |a| >= |b| per part
{
    const float2 s = __fadd2_rn(a, b);
    return dflt2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ dflt2 renorm2(dflt2 a) { return two_sum2(a.h, a.l); }

// a + b, low parts unnormalised (as add_lazy)
__device__ __forceinline__ dflt2 add_lazy2(dflt2 a, dflt2 b)
{
    const dflt2 s = two_sum2(a.h, b.h);
    return dflt2{s.h, __fadd2_rn(__fadd2_rn(a.l, b.l), s.l)};
}

// the error-free product of the leading parts plus the cross terms, for a
// double-float scalar m times both parts of a
__device__ __forceinline__ void mul2_parts(dflt2 a, dflt m, float2* p, float2* e)
{
    const float2 mh = f2s(m.h);
    *p = __fmul2_rn(a.h, mh);
    const float2 pn = __fmul2_rn(a.h, f2s(-m.h));                        // -p, exactly
    *e = __ffma2_rn(a.h, f2s(m.l), __ffma2_rn(a.l, mh, __ffma2_rn(a.h, mh, pn)));
}
// m a, normalised
__device__ __forceinline__ dflt2 mul2_df(dflt2 a, dflt m)
{
    float2 p, e;
    mul2_parts(a, m, &p, &e);
    return fast_two_sum2(p, e);
}
// acc + m b, low part unnormalised (as mac_lazy)
__device__ __forceinline__ dflt2 mac_lazy2(dflt2 acc, dflt m, dflt2 b)
{
    float2 p, e;
    mul2_parts(b, m, &p, &e);
    const dflt2 s = two_sum2(acc.h, p);
    return dflt2{s.h, __fadd2_rn(acc.l, __fadd2_rn(s.l, e))};
}

// the four passes of dfops.cuh on packed pairs (same grouping)
template <int P>
__device__ __forceinline__ void pascal_up2(dflt2* c)
{
#pragma unroll
    for (int g = 0; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j] = add_lazy2(c[j], c[j + 1]);
        }
    }
}
template <int P>
__device__ __forceinline__ void pascal_down2(dflt2* c)
{
#pragma unroll
    for (int g = 1; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4 && i < P; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j + 1] = add_lazy2(c[j + 1], c[j]);
        }
    }
}
template <int P>
__device__ __forceinline__ void pascal_up_mul2(dflt2* c, dflt a)
{
#pragma unroll
    for (int g = 0; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j] = mac_lazy2(c[j], a, c[j + 1]);
        }
    }
}
template <int P>
__device__ __forceinline__ void pascal_down_mul2(dflt2* c, dflt b)
{
#pragma unroll
    for (int g = 1; g < P; g += 4) {
#pragma unroll 1
        for (int i = g; i < g + 4 && i < P; ++i) {
#pragma unroll
            for (int j = P - 1; j >= g; --j)
                if (j >= i) c[j + 1] = mac_lazy2(c[j + 1], b, c[j]);
        }
    }
}

// coefficient l of a row (Re at 2l, Im at 2l + 1) as a packed pair, and back
__device__ __forceinline__ dflt2 ld_pair(const dflt* row, int l)
{
    const dflt re = row[2 * l], im = row[2 * l + 1];
    return dflt2{make_float2(re.h, im.h), make_float2(re.l, im.l)};
}
__device__ __forceinline__ void st_pair(dflt* row, int l, dflt2 v)
{
    row[2 * l] = dflt(v.h.x, v.l.x);
    row[2 * l + 1] = dflt(v.h.y, v.l.y);
}

}  // namespace sfmm
