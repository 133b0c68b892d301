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

}  // namespace sfmm
