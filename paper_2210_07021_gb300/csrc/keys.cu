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
#include "common.cuh"

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

__global__ void k_keys(const double* __restrict__ xyz, int64_t n, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ iota)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        keys[i] = key29(x, y, z);
        if (iota) iota[i] = (uint32_t)i;
    }
}

}  // namespace

cudaError_t launch_keys(const double* xyz, int64_t n, uint64_t* keys, uint32_t* iota, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_keys<<<(unsigned)blocks, 256, 0, s>>>(xyz, n, keys, iota); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
