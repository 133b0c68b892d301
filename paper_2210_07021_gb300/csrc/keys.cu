// Order-29 nested HEALPix keys of unit vectors (Sec. 3.1; Gorski et al. 2005).
//
// This file is compiled with -fmad=false: every operation below is a single
// correctly rounded IEEE double operation (+, -, *, /, sqrt) in a fixed order,
// so the keys are bit-identical to any other implementation that evaluates the
// same published formulas in the same order.
//
// Azimuth, in quarter turns: octant reduction to t = min(|x|,|y|)/max(|x|,|y|);
// atan(t) from the Gregory series sum (-1)^k t^(2k+1)/(2k+1) after the
// reductions t -> (t-1)/(t+1) (adds pi/4) when t > tan(pi/8) and the
// half-angle identity atan(t) = 2 atan(t/(1+sqrt(1+t^2))), leaving
// |t| <= tan(pi/16) where 12 terms reach double precision.
// ang2pix_nest: the equatorial / polar-cap formulas of Gorski et al. (2005),
// with 1 - |z| = (x^2 + y^2)/(1 + |z|) in the caps.
//
// Fast path.  The same quantities are first computed in double-float
// arithmetic on the FP32 pipe (about 46 significant bits; FP64 arithmetic on
// this GPU runs at 1/64 of the FP32 rate, so the fast path issues no FP64
// instruction at all: the coordinates are split into (hi, lo) FP32 pairs and
// compared through their bit patterns): the ratio by a double-float
// division, atan by a 129-entry table of atan(j/128) (rounded from the host's
// FP64 atan) and atan(r) = r - r^3/3 + r^5/5 - r^7/7 for |r| <= 1/256, then
// the equatorial or polar formula.  Every integer the key
// depends on is a floor of a non-negative value v (v = N_side (1/2 + tt -+ 3z/4),
// N_side tp sqrt(3(1-|z|)), ..., and tt itself in the caps); the fast path keeps
// floor(v) only when v lies at least KEY_MARGIN from an integer.  Both its own
// error and that of the FP64 routine are below 2^-16 in these units, so the
// floors then agree; otherwise the point takes the FP64 routine above.  The
// keys are therefore those of the FP64 routine, bit for bit.
#include "common.cuh"
#include "dfloat.cuh"

#include <cmath>

namespace sfmm {

namespace {

constexpr double TAN_PI_8 = 0.41421356237309503;
constexpr double TWO_OVER_PI = 0.6366197723675814;
constexpr double GREG0 = 1.0, GREG1 = -1.0 / 3.0, GREG2 = 1.0 / 5.0, GREG3 = -1.0 / 7.0,
                 GREG4 = 1.0 / 9.0, GREG5 = -1.0 / 11.0, GREG6 = 1.0 / 13.0, GREG7 = -1.0 / 15.0,
                 GREG8 = 1.0 / 17.0, GREG9 = -1.0 / 19.0, GREG10 = 1.0 / 21.0, GREG11 = -1.0 / 23.0;

__device__ __forceinline__ double atan_quarter_01(double t)
{
    const bool big = t > TAN_PI_8;
    const double t1 = big ? (t - 1.0) / (t + 1.0) : t;
    const double t2 = t1 / (1.0 + sqrt(1.0 + t1 * t1));
    const double s = t2 * t2;
    double p = GREG11;
    p = p * s + GREG10;
    p = p * s + GREG9;
    p = p * s + GREG8;
    p = p * s + GREG7;
    p = p * s + GREG6;
    p = p * s + GREG5;
    p = p * s + GREG4;
    p = p * s + GREG3;
    p = p * s + GREG2;
    p = p * s + GREG1;
    p = p * s + GREG0;
    const double a = (2.0 * t2) * p;
    const double v = a * TWO_OVER_PI;
    return big ? 0.5 + v : v;
}

__device__ __forceinline__ double phi_quarter(double x, double y)
{
    const double ax = fabs(x), ay = fabs(y);
    const bool swap = ay > ax;
    const double num = swap ? ax : ay;
    const double den = swap ? ay : ax;
    if (den == 0.0) return 0.0;
    const double u = atan_quarter_01(num / den);
    const double v = swap ? 1.0 - u : u;
    const bool xpos = x >= 0.0, ypos = y >= 0.0;
    double tt;
    if (xpos && ypos) tt = v;
    else if (!xpos && ypos) tt = 2.0 - v;
    else if (!xpos && !ypos) tt = 2.0 + v;
    else tt = 4.0 - v;
    return tt >= 4.0 ? tt - 4.0 : tt;
}

__device__ __forceinline__ uint64_t spread_bits(uint64_t v)
{
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

__device__ __forceinline__ uint64_t key29(double x, double y, double z)
{
    const int64_t ns = int64_t(1) << ORDER_MAX;
    const double nside = (double)ns;
    const double za = fabs(z);
    const double tt = phi_quarter(x, y);
    int64_t face, ix, iy;
    if (za <= 2.0 / 3.0) {
        const double temp1 = nside * (0.5 + tt);
        const double temp2 = nside * z * 0.75;
        const int64_t jp = (int64_t)(temp1 - temp2);
        const int64_t jm = (int64_t)(temp1 + temp2);
        const int64_t ifp = jp >> ORDER_MAX, ifm = jm >> ORDER_MAX;
        face = (ifp == ifm) ? (ifp | 4) : ((ifp < ifm) ? ifp : (ifm + 8));
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int64_t ntt = (int64_t)tt;
        if (ntt > 3) ntt = 3;
        const double tp = tt - (double)ntt;
        const double one_m_za = (x * x + y * y) / (1.0 + za);
        const double tmp = nside * sqrt(3.0 * one_m_za);
        int64_t jp = (int64_t)(tp * tmp);
        int64_t jm = (int64_t)((1.0 - tp) * tmp);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z > 0.0) { face = ntt; ix = ns - jm - 1; iy = ns - jp - 1; }
        else         { face = ntt + 8; ix = jp; iy = jm; }
    }
    return ((uint64_t)face << (2 * ORDER_MAX)) | spread_bits((uint64_t)ix) | (spread_bits((uint64_t)iy) << 1);
}

// ------------------------------------------------------------- fast path
constexpr float KEY_MARGIN = 1.0f / 16384.0f;

// Bit-pattern helpers: for finite doubles, |a| <= |b| exactly when the
// patterns with the sign cleared compare so as unsigned integers.
__device__ __forceinline__ uint64_t abs_bits(double v) { return (uint64_t)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull; }
__device__ __forceinline__ bool nonneg(double v)        // v >= 0.0 (true for -0.0 too)
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) == 0 || (b & 0x7FFFFFFFFFFFFFFFull) == 0;
}
// |v| as (hi, lo): hi = the leading 24 bits of the significand (truncated),
// lo = the remaining 29 bits rounded to FP32 (relative error 2^-47), built
// from the bit pattern without the FP64 pipe.  Values below 2^-60 give 0
// (the callers only need them to 2^-60 absolute).
__device__ __forceinline__ dflt dfl_abs_from_bits(uint64_t b)
{
    const int e = (int)(b >> 52) - 1023;
    if (e < -60) return dflt(0.f, 0.f);
    const uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const float hi = __int_as_float(((e + 127) << 23) | (int)((m >> 29) & 0x7FFFFF));
    const float lo = __fmul_rn(__int2float_rn((int)(m & 0x1FFFFFFF)), __int_as_float((e - 52 + 127) << 23));
    return dflt(hi, lo);
}
__device__ __forceinline__ dflt dfl_from_bits(double v)
{
    const dflt a = dfl_abs_from_bits(abs_bits(v));
    return nonneg(v) ? a : -a;
}

// floor of a double-float v >= 0 (|v| < 2^40); *ok = false when v is within
// KEY_MARGIN of an integer
__device__ __forceinline__ int64_t dfl_floor_checked(dflt v, bool* ok)
{
    const float fh = floorf(v.h);
    const float g = __fadd_rn(__fsub_rn(v.h, fh), v.l);    // fractional part, to 2^-24
    const float k = floorf(g);
    const float fr = __fsub_rn(g, k);
    if (fr < KEY_MARGIN || fr > 1.f - KEY_MARGIN) *ok = false;
    return (int64_t)__float2ll_rz(fh) + (int64_t)k;
}

__device__ __forceinline__ dflt dfl_sqrt_key(dflt a)
{
    const float s0 = sqrtf(a.h);
    // one Newton correction from the double-float residual a - s0^2
    const float p = __fmul_rn(s0, s0);
    const float e = __fmaf_rn(s0, s0, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), e), a.l);
    return dfl_fast_two_sum(s0, __fdiv_rn(r, __fadd_rn(s0, s0)));
}

struct KeyTables {
    float4 atan_c[129];    // atan(j/128) as (hi, lo), then (unused, unused)
    float4 two_over_pi;    // 2/pi as (hi, lo)
};

// Order-29 key by the double-float fast path; *ok = false when a floor decision
// is too close to call (the caller then uses key29).
__device__ __forceinline__ uint64_t key29_fast(double x, double y, double z, const KeyTables& kt, bool* ok)
{
    const int64_t ns = int64_t(1) << ORDER_MAX;
    const float nside = (float)ns;
    const uint64_t bx = abs_bits(x), by = abs_bits(y);
    const bool swap = by > bx;                                        // |y| > |x|
    const uint64_t bnum = swap ? bx : by, bden = swap ? by : bx;
    dflt tt(0.f, 0.f);
    // within 2^-60 of the axis the float conversions lose the ratio: FP64 routine
    if (bden != 0 && bden < (uint64_t(1023 - 60) << 52)) { *ok = false; return 0; }
    if (bden != 0) {
        const dflt T = dfl_abs_from_bits(bnum) / dfl_abs_from_bits(bden);   // t in [0, 1]
        const int j = min(128, max(0, (int)__fadd_rn(__fmul_rn(T.h, 128.f), 0.5f)));
        const float c = (float)j * (1.f / 128.f);
        // r = (t - c) / (1 + t c), |r| <= 1/256: atan t = atan c + atan r
        const dflt R = (T - dflt(c, 0.f)) / (dflt(1.f, 0.f) + T * c);
        const float rh = R.h, s2 = __fmul_rn(rh, rh);
        const float tail = __fmul_rn(__fmul_rn(rh, s2), -1.f / 3.f + s2 * (0.2f - s2 * (1.f / 7.f)));
        const float4 a = kt.atan_c[j];
        const dflt A = dflt(a.x, a.y) + (R + dflt(tail, 0.f));
        const dflt u = A * dflt(kt.two_over_pi.x, kt.two_over_pi.y);   // quarter turns, [0, 1/2]
        const dflt v = swap ? dflt(1.f, 0.f) - u : u;
        const bool xpos = nonneg(x), ypos = nonneg(y);
        if (xpos && ypos) tt = v;
        else if (!xpos && ypos) tt = dflt(2.f, 0.f) - v;
        else if (!xpos && !ypos) tt = dflt(2.f, 0.f) + v;
        else tt = dflt(4.f, 0.f) - v;
        // tt wraps from 4 to 0 at phi = 2 pi: too close to the wrap, let the FP64 routine decide
        if (__fsub_rn(4.f, tt.h) < 1.f / 1073741824.f) *ok = false;
        if (tt.h >= 4.f) tt = tt - dflt(4.f, 0.f);
    }
    const uint64_t bz = abs_bits(z);
    int64_t face, ix, iy;
    if (bz <= 0x3FE5555555555555ull) {                               // |z| <= 2/3 (the FP64 constant)
        const dflt W = dflt(0.5f, 0.f) + tt;
        const dflt Z = dfl_from_bits(z) * 0.75f;
        const int64_t jp = dfl_floor_checked((W - Z) * nside, ok);
        const int64_t jm = dfl_floor_checked((W + Z) * nside, ok);
        const int64_t ifp = jp >> ORDER_MAX, ifm = jm >> ORDER_MAX;
        face = (ifp == ifm) ? (ifp | 4) : ((ifp < ifm) ? ifp : (ifm + 8));
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int64_t ntt = dfl_floor_checked(tt * nside, ok) >> ORDER_MAX;   // floor(tt), decided at N_side resolution
        if (ntt > 3) ntt = 3;
        const dflt tp = tt - dflt((float)ntt, 0.f);
        const dflt X = dfl_abs_from_bits(bx), Y = dfl_abs_from_bits(by);
        const dflt one_m_za = (X * X + Y * Y) / (dflt(1.f, 0.f) + dfl_abs_from_bits(bz));
        const dflt tmp = dfl_sqrt_key(one_m_za * 3.f) * nside;
        int64_t jp = dfl_floor_checked(tp * tmp, ok);
        int64_t jm = dfl_floor_checked((dflt(1.f, 0.f) - tp) * tmp, ok);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (bz != 0 && nonneg(z)) { face = ntt; ix = ns - jm - 1; iy = ns - jp - 1; }   // z > 0
        else                      { face = ntt + 8; ix = jp; iy = jm; }
    }
    return ((uint64_t)face << (2 * ORDER_MAX)) | spread_bits((uint64_t)ix) | (spread_bits((uint64_t)iy) << 1);
}

__global__ void k_keys(const double* __restrict__ xyz, int64_t n, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ iota, KeyTables kt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        bool ok = true;
        uint64_t k = key29_fast(x, y, z, kt, &ok);
        if (!ok) k = key29(x, y, z);
        keys[i] = k;
        if (iota) iota[i] = (uint32_t)i;
    }
}

KeyTables make_key_tables()
{
    KeyTables kt;
    for (int j = 0; j <= 128; ++j) {
        const double a = std::atan(j / 128.0);
        const float h = (float)a;
        kt.atan_c[j] = make_float4(h, (float)(a - (double)h), 0.f, 0.f);
    }
    const double tp = 2.0 / 3.14159265358979323846;
    const float h = (float)tp;
    kt.two_over_pi = make_float4(h, (float)(tp - (double)h), 0.f, 0.f);
    return kt;
}

}  // namespace

cudaError_t launch_keys(const double* xyz, int64_t n, uint64_t* keys, uint32_t* iota, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    static const KeyTables kt = make_key_tables();
    k_keys<<<(unsigned)blocks, 256, 0, s>>>(xyz, n, keys, iota, kt); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
