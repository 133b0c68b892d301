// M2L (Lemma 3) in double-float, one thread per FMM-act pair: the
// translation of the 1e-6 and 1e-10 paths (precision SFMM_MIXED and
// SFMM_MIXED_DF), whose far field is carried in double-float.
//
// In the scaled frames of expand.cu, with u~_l = (a ph1)^l X_l and
// rho = g/(a b) = 1/cos^2(theta/2), Lemma 3 becomes
//     t_n = sum_{l >= n} C(l, n) u~_l                       (n = 0..p)
//     o_l = sum_{n <= l} C(l-1, n-1) rho^n t_n              (l = 1..p)
//     Y_l = (b ph2)^l (-Q/l + o_l),   C' = C + 2 Q log sin(theta/2) + 2 Re t_0,   Q' = Q.
// Both binomial sums are synthetic-division passes made of additions only:
// the Taylor shift by one (for i < p, for j = p-1 down to i: c_j += c_{j+1})
// turns u~ into t, and its dual (for i = 1..p-1, for j = p-1 down to i:
// x_j += x_{j-1}) turns x_m = rho^{m+1} t_{m+1} into x_m = o_{m+1}.  That is
// p^2 double-float additions per component and pair, with the diagonal
// scalings (powers of a ph1, rho and b ph2) as O(p) double-float products:
// no binomial table, no shuffles, every value in the thread's registers.
//
// The pairs arrive grouped by target box.  Each warp takes 32 consecutive
// pairs, stages their outputs in shared memory (one row per pair), and each
// lane then sums one coefficient column over the runs of equal target and
// adds the run sums to an FP64 accumulator per target box (atomicAdd on
// float64 carries 53 bits, above the 48 of double-float).  Pairs with rho > 8.7
// (centres at or near antipodes: rho^32 would exceed 2^100, and a b = 0 at
// exact antipodes) are listed for the warp kernel of expand.cu, which uses a,
// b and g directly.
#include "common.cuh"
#include "dfloat.cuh"
#include "xgeo.cuh"
#include "dfops.cuh"

namespace sfmm {

namespace {

constexpr int PW = 4;            // warps per CTA

// P: the order rounded up to a multiple of 4 (orders p+1..P are zero and cost
// only their additions).  Each thread's row (2P + 3 double-floats in shared
// memory) holds the pair's scaled vector between the steps and then its
// output.  The two binomial passes are unrolled once and run for the real and
// then the imaginary part (a runtime loop), with the part in registers; the
// O(p) diagonal steps are runtime loops.  This keeps the code within the
// instruction cache and the registers at five CTAs per SM for p <= 20 (the
// packed FP32x2 form of updown_df.cu measured slower here: it needs twice the
// registers and the FMA pipe, not the issue rate, bounds this kernel).
template <int P>
__global__ void __launch_bounds__(128, (P <= 20 ? 5 : P <= 24 ? 4 : 3))
k_m2l_pair(int64_t n_cap, const int64_t* d_n, const uint64_t* __restrict__ ptgt, const uint32_t* __restrict__ psrc,
                                                  const XGeoRho* __restrict__ geo, const dflt* __restrict__ mpole,
                                                  int p, double* __restrict__ acc, uint32_t* __restrict__ leftover,
                                                  uint32_t* __restrict__ n_left)
{
    constexpr int RS = 2 * P + 3;                 // row stride (odd: conflict-free row access)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_tgt[PW][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    dflt* rows = reinterpret_cast<dflt*>(smem_raw) + (size_t)wid * 32 * RS;
    dflt* row = rows + lane * RS;
    const int ncol = 2 * p + 2;
    const int64_t n_pairs = dcount(d_n, n_cap);
    const int64_t stride = (int64_t)gridDim.x * PW * 32;
    for (int64_t base = ((int64_t)blockIdx.x * PW + wid) * 32; base < n_pairs; base += stride) {
        const int64_t k = base + lane;
        const bool valid = k < n_pairs;
        int tnode = -1;
        bool big = true;
        XGeoRho G;
        if (valid) {
            G = geo[k];
            tnode = (int)ptgt[k];
            big = G.big != 0;
            if (big) leftover[atomicAdd(n_left, 1u)] = (uint32_t)k;
        }
        if (!big) {
            const dflt* e = mpole + (size_t)psrc[k] * EXP_STRIDE;
            dflt Q;
            const dflt C = ld_dflt2(e, &Q);
            // u~_l = (a ph1)^l X_l into the row (zero for p < l <= P)
            {
                dflt zr = G.ar, zi = G.ai;
#pragma unroll 1
                for (int l = 1; l <= P; ++l) {
                    if (l > 1) {
                        dflt nr, ni;
                        cmul_df(zr, zi, G.ar, G.ai, &nr, &ni);
                        zr = nr;
                        zi = ni;
                    }
                    dflt ur(0.f, 0.f), ui(0.f, 0.f);
                    if (l <= p) {
                        dflt xi;
                        const dflt xr = ld_dflt2(e + 2 * l, &xi);
                        cmul_df(zr, zi, xr, xi, &ur, &ui);
                    }
                    row[2 * l] = ur;
                    row[2 * l + 1] = ui;
                }
            }
            // both binomial stages, for the real and then the imaginary part (one unrolled copy)
            dflt t0(0.f, 0.f);
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
                dflt c[P + 1];
                c[0] = dflt(0.f, 0.f);
#pragma unroll
                for (int l = 1; l <= P; ++l) c[l] = row[2 * l + part];
                pascal_up<P>(c);                  // t = B2 u~: the Taylor shift by one
                if (part == 0) t0 = renorm(c[0]);
                // x_m = rho^(m+1) t_(m+1), kept at index m + 1
                dflt rp = G.rho;
#pragma unroll
                for (int n = 1; n <= P; ++n) {
                    c[n] = renorm(c[n]) * rp;
                    if (n < P) rp = rp * G.rho;
                }
                pascal_down<P>(c);                // o = B1 x: the dual pass
#pragma unroll
                for (int l = 1; l <= P; ++l) row[2 * l + part] = renorm(c[l]);
            }
            // C' = C + 2 Q log sin(theta/2) + 2 Re t_0,  Q' = Q
            const dflt two(2.f, 0.f);
            row[0] = C + two * (Q * G.logk + t0);
            row[1] = Q;
            // Y_l = (b ph2)^l (-Q/l + o_l)
            {
                dflt zr = G.br, zi = G.bi;
#pragma unroll 1
                for (int l = 1; l <= p; ++l) {
                    if (l > 1) {
                        dflt nr, ni;
                        cmul_df(zr, zi, G.br, G.bi, &nr, &ni);
                        zr = nr;
                        zi = ni;
                    }
                    const float fl = (float)l, il = 1.f / fl;
                    const float q1 = __fmul_rn(Q.h, il);                       // Q / l: leading quotient
                    const float rq = __fadd_rn(__fmaf_rn(-q1, fl, Q.h), Q.l);  // and one correction
                    const dflt ql = dfl_fast_two_sum(q1, __fmul_rn(rq, il));
                    const dflt orr = row[2 * l] - ql, oi = row[2 * l + 1];
                    cmul_df(zr, zi, orr, oi, &row[2 * l], &row[2 * l + 1]);
                }
            }
        } else {
            for (int c = 0; c < ncol; ++c) row[c] = dflt(0.f, 0.f);
        }
        s_tgt[wid][lane] = tnode;
        __syncwarp();
        // per-target run sums of each coefficient column, added to the FP64 accumulators
        const int nrows = n_pairs - base < 32 ? (int)(n_pairs - base) : 32;
        for (int c = lane; c < ncol; c += 32) {
            int cur = s_tgt[wid][0];
            dflt a(0.f, 0.f);
            for (int r = 0; r < nrows; ++r) {
                const int t = s_tgt[wid][r];
                if (t != cur) {
                    atomicAdd(acc + (size_t)cur * EXP_STRIDE + c, (double)a.h + (double)a.l);
                    a = dflt(0.f, 0.f);
                    cur = t;
                }
                a = add_lazy(a, rows[r * RS + c]);
            }
            atomicAdd(acc + (size_t)cur * EXP_STRIDE + c, (double)a.h + (double)a.l);
        }
        __syncwarp();
    }
}

template <int P>
cudaError_t launch_p(int64_t n_pairs, const int64_t* d_n, const uint64_t* ptgt, const uint32_t* psrc,
                     const XGeoRho* geo, const dflt* mpole, int p, double* acc, uint32_t* leftover, uint32_t* n_left,
                     cudaStream_t s)
{
    const size_t smem = (size_t)PW * 32 * (2 * P + 3) * sizeof(dflt);
    cudaError_t e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaFuncSetAttribute(k_m2l_pair<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
        (e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_m2l_pair<P>, PW * 32, smem)))
        return e;
    const int64_t chunks = (n_pairs + PW * 32 - 1) / (PW * 32);
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t grid = chunks < cap ? chunks : cap;
    k_m2l_pair<P><<<(unsigned)grid, PW * 32, smem, s>>>(n_pairs, d_n, ptgt, psrc, geo, mpole, p, acc, leftover, n_left);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_m2l_pair(int64_t n_pairs, const int64_t* d_n, const uint64_t* ptgt, const uint32_t* psrc, const void* geo,
                            const void* mpole, int p, double* acc, uint32_t* leftover, uint32_t* n_left,
                            cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    const XGeoRho* G = static_cast<const XGeoRho*>(geo);
    const dflt* mp = static_cast<const dflt*>(mpole);
    switch ((p + 3) / 4 * 4) {
    case 4: return launch_p<4>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 8: return launch_p<8>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 12: return launch_p<12>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 16: return launch_p<16>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 20: return launch_p<20>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 24: return launch_p<24>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 28: return launch_p<28>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    case 32: return launch_p<32>(n_pairs, d_n, ptgt, psrc, G, mp, p, acc, leftover, n_left, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfmm
