// Evaluation at the targets (Sec. 3.6): L2P of the leaf's local expansion plus
// the near-field direct sum over the leaf's direct-act list, FP64.
//
// Far field, in the leaf frame with w = z(theta^(L), phi^(L)) = u + i v and
// F(w) = sum_l A_l w^l:
//   psi_e = C + Q log(1 + cos theta) + 2 Re F(w)
//   alpha_u - i alpha_v = (1 + |w|^2) F'(w) - Q conj(w)
// where (alpha_u, alpha_v) are the components on the unit vectors of the
// w-chart at the target, e_u = e_theta(L) - u (c + x), e_v = e_phi(L) - v (c + x).
// Along the radial direction this is the printed
//   alpha_theta^(L) = -Q tan(theta/2) + 2 Re sum (l / sin theta) A_l z^l,
// and it stays regular at w = 0.
//
// Near field (Eq. SUM with Eq. GRE_FUN and its gradient, Eq. ALP_PSI):
//   psi_i   = (1/4pi) sum_j q_j [log d_j^2 - log 4]
//   alpha_i = (1/2pi) [ sum_j q_j (x - y_j) / d_j^2 - (x/2) sum_j q_j ]
// with d^2 = |x - y|^2 from coordinate differences; d^2 == 0 pairs are skipped.
//
// One warp per target leaf.  The leaf's targets are taken in groups of tpw,
// the largest power of two not above the targets left (at most 32), so that
// no lane idles; each target of a group gets 32/tpw lanes that split its
// sources and are combined by xor shuffles.  (The FP32 kernel, whose pair loop
// is cheap next to restaging its sources per group, keeps one group size per
// leaf: the power of two not below the leaf's targets.)
#include "common.cuh"
#include "dfloat.cuh"
#include "xgeo.cuh"

#include <cmath>

namespace sfmm {

namespace {

constexpr double INV4PI = 0.079577471545947667884;
constexpr double PI = 3.14159265358979323846;
constexpr double INV2PI = 0.15915494309189533577;
constexpr double LOG2 = 0.69314718055994530942;
constexpr double LOG4 = 1.3862943611198906188;
constexpr float FLT_MIN_F = 1.17549435e-38f;     // the smallest normal FP32 number
constexpr float LN2_H = 0.693147182464599609375f;   // log 2 rounded to FP32
constexpr float LN2_L = -1.9046542121259336e-09f;   // log 2 - LN2_H
constexpr float INV4PI_H = (float)INV4PI;             // 1/(4 pi) as a double-float
constexpr float INV4PI_L = (float)(INV4PI - (double)INV4PI_H);

struct EvalArgs {
    TreeView T;
    const int* leaves;        // target leaves (tcount > 0)
    int64_t n_leaves;
    const int64_t* d_n_leaves;      // graph mode: the leaf count on the device (n_leaves: the capacity)
    const double4_32a* src;       // key-sorted sources (x, y, z, q)
    const double4_32a* tgt;       // key-sorted targets (x, y, z, -)
    const uint32_t* tperm;    // original index of each sorted target
    const int64_t* p2p_off;
    const uint32_t* p2p_src;
    const double* local;
    const double* base_mpole; // multipoles of the 12 base boxes (for the zero-mean shift)
    int p;
    int want_psi;
    int zero_mean;
    double* psi;
    double* alpha;
    double* gamma;            // [M][2] shear (gamma_1, gamma_2) in (e_theta, e_phi), or NULL
    double* mu;               // [M] magnification 1/((1 - tr H/2)^2 - |gamma|^2), or NULL (with gamma)
    unsigned long long* leaf_ctr;   // zero at launch: the warps take target leaves from it one at a time
    double npm_s;             // Near Particle Model: sin^2(sigma/2) (NPM kernels only)
};

__device__ __forceinline__ double group_sum(double v, int lpt)
{
    for (int o = lpt >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// SHEAR: also the trace-free part of the covariant Hessian (Sec. 2.2, Eq.
// GAM_DEF).  Near field: H_ab = -(e_a.d)(e_b.d)/(pi d^4) + (isotropic), so the
// shear needs S = sum q d d^T / d^4.  Far field, in the leaf chart w with
// metric lambda^2 |dw|^2, lambda = 2/(1 + |w|^2):
//   (H_uu - H_vv)/2 - i H_uv = (2/lambda^2) [d_w^2 f - 2 (d_w log lambda) d_w f]
//                            = ((1 + |w|^2)^2 / 2) [F'' + 2 conj(w) F' / (1 + |w|^2)] - Q conj(w)^2 / 2
// for f = C + Q log(1 + cos theta) + 2 Re F(w) (conformal Christoffel symbols;
// 1 + cos theta = 2/(1 + |w|^2)); (H_uu, H_vv, H_uv) on the chart's unit
// vectors e_u, e_v are then projected onto (e_theta, e_phi) at the target.
//
// NPM: pairs closer than the particle radius (u = d^2/4 < s = sin^2(sigma/2))
// use the smoothed particle (Secs. 3.2, 4.2): alpha scaled by
// f = (m(u) - u)/(1 - u), m = 2u/s - u^2/s^2 (Gauss's law on the sphere), and
// log u replaced by log s - (1 - u/s) + ((1 - s)^2/s^2)(log1p(t) - t),
// t = (s - u)/(1 - s) (the point-mass potential continued into the cap).
// The next target leaf of a warp, taken from a global counter by lane 0.
__device__ __forceinline__ int64_t next_leaf(unsigned long long* ctr, int lane)
{
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(ctr, 1ull);
    return (int64_t)__shfl_sync(FULL, w, 0);
}

template <bool SHEAR, bool NPM>
__global__ void __launch_bounds__(128) k_eval(EvalArgs A)
{
    const int lane = threadIdx.x & 31;
    double shift = 0.0, qtot = 0.0;        // qtot = sum q / 4pi (the base boxes' Q)
    for (int b = 0; b < 12; ++b) qtot += A.base_mpole[(size_t)b * EXP_STRIDE + 1];
    if (A.zero_mean) shift = qtot;
    for (;;) {
        const int64_t w = next_leaf(A.leaf_ctr, lane);
        if (w >= dcount(A.d_n_leaves, A.n_leaves)) break;
        const int leaf = A.leaves[w];
        const int tf = A.T.tfirst[leaf], tc = A.T.tcount[leaf];
        const double* g = A.T.geom + (size_t)leaf * GEOM_STRIDE;
        const double* L = A.local + (size_t)leaf * EXP_STRIDE;
        const int64_t nb0 = A.p2p_off[leaf], nb1 = A.p2p_off[leaf + 1];
        for (int tb = 0, tpw = 0; tb < tc; tb += tpw) {
            tpw = min(32, 1 << (31 - __clz(tc - tb)));     // largest power of two <= the targets left
            const int lpt = 32 / tpw;
            const int slot = lane / lpt, sub = lane % lpt;
            const int ti = tb + slot;
            const bool active = ti < tc;
            const double4_32a x = A.tgt[tf + (active ? ti : 0)];
            double sl = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, sq = 0.0;
            double Sxx = 0.0, Syy = 0.0, Szz = 0.0, Sxy = 0.0, Sxz = 0.0, Syz = 0.0;
            double sqs = 0.0;                 // SHEAR: masses at the target's position (left out)
            double sqa = 0.0;                 // NPM: sum of f q (the alpha part of sum q)
            for (int64_t k = nb0; k < nb1; ++k) {
                const int sleaf = (int)A.p2p_src[k];
                const int f = A.T.first[sleaf], n = A.T.count[sleaf];
                for (int j = f + sub; j < f + n; j += lpt) {
                    const double4_32a y = A.src[j];
                    const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    if (NPM && d2 > 0.0) {
                        const double s = A.npm_s, u = 0.25 * d2;
                        double f = 1.0, lg;
                        if (u < s) {
                            const double m = 2.0 * u / s - u * u / (s * s);
                            f = (m - u) / (1.0 - u);
                            const double t = (s - u) / (1.0 - s);
                            lg = LOG4 + log(s) - (1.0 - u / s) + (1.0 - s) * (1.0 - s) / (s * s) * (log1p(t) - t);
                        } else {
                            lg = log(d2);
                        }
                        const double wq = f * y.w / d2;
                        sx += wq * dx;
                        sy += wq * dy;
                        sz += wq * dz;
                        sq += y.w;
                        sqa += f * y.w;
                        if (A.want_psi) sl += y.w * lg;
                    } else if (d2 > 0.0) {
                        const double wq = y.w / d2;
                        sx += wq * dx;
                        sy += wq * dy;
                        sz += wq * dz;
                        sq += y.w;
                        if (A.want_psi) sl += y.w * log(d2);
                        if (SHEAR) {
                            const double w4 = wq / d2;
                            Sxx += w4 * dx * dx; Syy += w4 * dy * dy; Szz += w4 * dz * dz;
                            Sxy += w4 * dx * dy; Sxz += w4 * dx * dz; Syz += w4 * dy * dz;
                        }
                    } else if (SHEAR) {
                        sqs += y.w;
                    }
                }
            }
            sx = group_sum(sx, lpt);
            sy = group_sum(sy, lpt);
            sz = group_sum(sz, lpt);
            sq = group_sum(sq, lpt);
            if (NPM) sqa = group_sum(sqa, lpt);
            else sqa = sq;
            if (A.want_psi) sl = group_sum(sl, lpt);
            if (SHEAR) {
                Sxx = group_sum(Sxx, lpt); Syy = group_sum(Syy, lpt); Szz = group_sum(Szz, lpt);
                Sxy = group_sum(Sxy, lpt); Sxz = group_sum(Sxz, lpt); Syz = group_sum(Syz, lpt);
                sqs = group_sum(sqs, lpt);
            }
            if (!active || sub != 0) continue;
            // ---- L2P in the leaf frame
            const double Dx = x.x - g[0], Dy = x.y - g[1], Dz = x.z - g[2];
            const double D2 = Dx * Dx + Dy * Dy + Dz * Dz;
            const double den = 2.0 - 0.5 * D2;                  // 1 + x.c
            const double wu = (Dx * g[3] + Dy * g[4] + Dz * g[5]) / den;
            const double wv = (Dx * g[6] + Dy * g[7] + Dz * g[8]) / den;
            const double inv_r = 1.0 / g[10];
            const cd om = mk(wu * inv_r, wv * inv_r);
            cd f = mk(0.0, 0.0), fd = mk(0.0, 0.0), fdd = mk(0.0, 0.0);
            for (int l = A.p; l >= 1; --l) {
                const cd a = mk(L[2 * l], L[2 * l + 1]);
                f = cadd(cmul(f, om), a);
                fd = cadd(cmul(fd, om), cscale(a, (double)l));
                if (SHEAR && l >= 2) fdd = cadd(cmul(fdd, om), cscale(a, (double)(l * (l - 1))));
            }
            const cd F = cmul(f, om);
            const cd Fp = cscale(fd, inv_r);                    // dF/dw
            const double C = L[0], Q = L[1];
            const double w2 = wu * wu + wv * wv;
            const double au = (1.0 + w2) * Fp.x - Q * wu;
            const double av = -(1.0 + w2) * Fp.y - Q * wv;
            const double cxx = g[0] + x.x, cyy = g[1] + x.y, czz = g[2] + x.z;
            double a3x = au * (g[3] - wu * cxx) + av * (g[6] - wv * cxx);
            double a3y = au * (g[4] - wu * cyy) + av * (g[7] - wv * cyy);
            double a3z = au * (g[5] - wu * czz) + av * (g[8] - wv * czz);
            // ---- near field
            a3x += INV2PI * (sx - 0.5 * x.x * sqa);
            a3y += INV2PI * (sy - 0.5 * x.y * sqa);
            a3z += INV2PI * (sz - 0.5 * x.z * sqa);
            const double rho = sqrt(x.x * x.x + x.y * x.y);
            double cp = 1.0, sp = 0.0;
            if (rho > 0.0) { cp = x.x / rho; sp = x.y / rho; }
            const uint32_t o = A.tperm[tf + ti];
            if (A.alpha) {
                A.alpha[2 * (size_t)o] = a3x * (x.z * cp) + a3y * (x.z * sp) - a3z * rho;
                A.alpha[2 * (size_t)o + 1] = -a3x * sp + a3y * cp;
            }
            if (A.want_psi) {
                const double psi_e = C + Q * (LOG2 + log1p(-0.25 * D2)) + 2.0 * F.x;
                A.psi[o] = psi_e + INV4PI * (sl - LOG4 * sq) + shift;
            }
            if (SHEAR) {
                // far field: chart-frame trace-free Hessian, then onto (e_theta, e_phi)
                const cd Fpp = cscale(fdd, inv_r * inv_r);
                const double opw = 1.0 + w2;
                const cd wb = mk(wu, -wv);
                const cd t1 = cadd(Fpp, cscale(cmul(wb, Fp), 2.0 / opw));
                const cd wb2 = cmul(wb, wb);
                const double gr = 0.5 * opw * opw * t1.x - 0.5 * Q * wb2.x;
                const double gi = 0.5 * opw * opw * t1.y - 0.5 * Q * wb2.y;
                const double huu = gr, huv = -gi;                        // H_vv = -H_uu (trace-free part)
                const double eux = g[3] - wu * cxx, euy = g[4] - wu * cyy, euz = g[5] - wu * czz;
                const double evx = g[6] - wv * cxx, evy = g[7] - wv * cyy, evz = g[8] - wv * czz;
                const double etx = x.z * cp, ety = x.z * sp, etz = -rho, epx = -sp, epy = cp;
                const double c1 = eux * etx + euy * ety + euz * etz, s1 = eux * epx + euy * epy;
                const double c2 = evx * etx + evy * ety + evz * etz, s2 = evx * epx + evy * epy;
                double g1 = 0.5 * (huu * (c1 * c1 - s1 * s1 - c2 * c2 + s2 * s2)) + huv * (c1 * c2 - s1 * s2);
                double g2 = huu * (c1 * s1 - c2 * s2) + huv * (c1 * s2 + c2 * s1);
                // near field: -(e_a^T S e_b)/pi
                const double stt = etx * (Sxx * etx + Sxy * ety + Sxz * etz) + ety * (Sxy * etx + Syy * ety + Syz * etz) +
                                   etz * (Sxz * etx + Syz * ety + Szz * etz);
                const double spp = epx * (Sxx * epx + Sxy * epy) + epy * (Sxy * epx + Syy * epy);
                const double stp = epx * (Sxx * etx + Sxy * ety + Sxz * etz) + epy * (Sxy * etx + Syy * ety + Syz * etz);
                g1 -= 0.5 * (stt - spp) / PI;
                g2 -= stp / PI;
                A.gamma[2 * (size_t)o] = g1;
                A.gamma[2 * (size_t)o + 1] = g2;
                if (A.mu) {       // tr H = kappa - kappa_bar = -(sum q of the masses not at x) / 4pi
                    const double trh = -qtot + INV4PI * sqs;
                    const double a = 1.0 - 0.5 * trh;
                    A.mu[o] = 1.0 / (a * a - g1 * g1 - g2 * g2);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Adjoint evaluation (FP64): the field of charges h_j (src.w) and tangent
// dipoles g_j (dip) at the sources, at the targets: Phi = psi-like sum plus
//   sum_j g_j . (y_j - x) / (2 pi r^2)                        (dipole potential)
// and its covariant gradient, the L2P part as in k_eval plus, per near pair,
//   P_x [ h_j (x - y_j) / (2 pi r^2) + ( -g_j / r^2 - 2 (g_j . (y_j - x)) (x - y_j) / r^4 ) / (2 pi) ].
// Writes Phi (if phi) and w_i times the gradient 3-vector (if grad3), at the
// caller's index of each target; w is float32 when w_f32.
struct EvalAdjArgs {
    EvalArgs E;
    const double4_32a* dip;   // key-sorted tangent dipoles (gx, gy, gz, -)
    const void* w;
    int w_f32;
    double* grad3;
};

__global__ void __launch_bounds__(128) k_eval_adj(EvalAdjArgs AA)
{
    const EvalArgs& A = AA.E;
    const int lane = threadIdx.x & 31;
    double shift = 0.0;
    if (A.zero_mean)
        for (int b = 0; b < 12; ++b) shift += A.base_mpole[(size_t)b * EXP_STRIDE + 1];
    for (;;) {
        const int64_t w = next_leaf(A.leaf_ctr, lane);
        if (w >= dcount(A.d_n_leaves, A.n_leaves)) break;
        const int leaf = A.leaves[w];
        const int tf = A.T.tfirst[leaf], tc = A.T.tcount[leaf];
        const double* g = A.T.geom + (size_t)leaf * GEOM_STRIDE;
        const double* L = A.local + (size_t)leaf * EXP_STRIDE;
        const int64_t nb0 = A.p2p_off[leaf], nb1 = A.p2p_off[leaf + 1];
        for (int tb = 0, tpw = 0; tb < tc; tb += tpw) {
            tpw = min(32, 1 << (31 - __clz(tc - tb)));
            const int lpt = 32 / tpw;
            const int slot = lane / lpt, sub = lane % lpt;
            const int ti = tb + slot;
            const double4_32a x = A.tgt[tf + ti];
            double sl = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, sq = 0.0;     // charges (as k_eval)
            double sd = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;               // dipoles
            for (int64_t k = nb0; k < nb1; ++k) {
                const int sleaf = (int)A.p2p_src[k];
                const int f = A.T.first[sleaf], n = A.T.count[sleaf];
                for (int j = f + sub; j < f + n; j += lpt) {
                    const double4_32a y = A.src[j];
                    const double4_32a gd = AA.dip[j];
                    const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 > 0.0) {
                        const double inv = 1.0 / d2;
                        const double wq = y.w * inv;
                        sx += wq * dx;
                        sy += wq * dy;
                        sz += wq * dz;
                        sq += y.w;
                        if (A.want_psi) sl += y.w * log(d2);
                        const double ge = -(gd.x * dx + gd.y * dy + gd.z * dz);   // g . (y - x)
                        sd += ge * inv;
                        const double c2 = -2.0 * ge * inv * inv;
                        vx += c2 * dx - gd.x * inv;
                        vy += c2 * dy - gd.y * inv;
                        vz += c2 * dz - gd.z * inv;
                    }
                }
            }
            sx = group_sum(sx, lpt);
            sy = group_sum(sy, lpt);
            sz = group_sum(sz, lpt);
            sq = group_sum(sq, lpt);
            sd = group_sum(sd, lpt);
            vx = group_sum(vx, lpt);
            vy = group_sum(vy, lpt);
            vz = group_sum(vz, lpt);
            if (A.want_psi) sl = group_sum(sl, lpt);
            if (sub != 0) continue;
            const double Dx = x.x - g[0], Dy = x.y - g[1], Dz = x.z - g[2];
            const double D2 = Dx * Dx + Dy * Dy + Dz * Dz;
            const double den = 2.0 - 0.5 * D2;
            const double wu = (Dx * g[3] + Dy * g[4] + Dz * g[5]) / den;
            const double wv = (Dx * g[6] + Dy * g[7] + Dz * g[8]) / den;
            const double inv_r = 1.0 / g[10];
            const cd om = mk(wu * inv_r, wv * inv_r);
            cd f = mk(0.0, 0.0), fd = mk(0.0, 0.0);
            for (int l = A.p; l >= 1; --l) {
                const cd a = mk(L[2 * l], L[2 * l + 1]);
                f = cadd(cmul(f, om), a);
                fd = cadd(cmul(fd, om), cscale(a, (double)l));
            }
            const cd F = cmul(f, om);
            const cd Fp = cscale(fd, inv_r);
            const double C = L[0], Q = L[1];
            const double w2 = wu * wu + wv * wv;
            const double au = (1.0 + w2) * Fp.x - Q * wu;
            const double av = -(1.0 + w2) * Fp.y - Q * wv;
            const double cxx = g[0] + x.x, cyy = g[1] + x.y, czz = g[2] + x.z;
            double a3x = au * (g[3] - wu * cxx) + av * (g[6] - wv * cxx);
            double a3y = au * (g[4] - wu * cyy) + av * (g[7] - wv * cyy);
            double a3z = au * (g[5] - wu * czz) + av * (g[8] - wv * czz);
            // near field: charges (projected form of k_eval) + dipoles projected by P_x
            const double xv = x.x * vx + x.y * vy + x.z * vz;
            a3x += INV2PI * (sx - 0.5 * x.x * sq + vx - xv * x.x);
            a3y += INV2PI * (sy - 0.5 * x.y * sq + vy - xv * x.y);
            a3z += INV2PI * (sz - 0.5 * x.z * sq + vz - xv * x.z);
            const uint32_t o = A.tperm[tf + ti];
            if (AA.grad3) {
                const double wt = AA.w_f32 ? (double)static_cast<const float*>(AA.w)[o]
                                           : static_cast<const double*>(AA.w)[o];
                AA.grad3[3 * (size_t)o] = wt * a3x;
                AA.grad3[3 * (size_t)o + 1] = wt * a3y;
                AA.grad3[3 * (size_t)o + 2] = wt * a3z;
            }
            if (A.want_psi) {
                const double psi_e = C + Q * (LOG2 + log1p(-0.25 * D2)) + 2.0 * F.x;
                A.psi[o] = psi_e + INV4PI * (sl - LOG4 * sq) + INV2PI * sd + shift;
            }
        }
    }
}

__global__ void k_count_pairs(TreeView T, const int* __restrict__ leaves, int64_t n, const int64_t* __restrict__ off,
                              const uint32_t* __restrict__ src, unsigned long long* __restrict__ out)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x) {
        const int leaf = leaves[w];
        unsigned long long c = 0;
        for (int64_t k = off[leaf]; k < off[leaf + 1]; ++k) c += (unsigned long long)T.count[src[k]];
        atomicAdd(out, c * (unsigned long long)T.tcount[leaf]);
    }
}

// ------------------------------------------------------------------------
// Mixed-precision evaluation.  Every offset is carried as an FP32 pair
// (hi + lo, lo = the FP64 remainder), so differences of nearby points keep
// their relative accuracy without FP64 arithmetic in the pair loop:
//   source offset from the target leaf centre =
//       (offset from its own leaf centre, formed once per source in FP64)
//     + (offset between the two leaf centres, one FP64 difference per near
//        leaf, taken lane-parallel), added by an error-free two-sum;
//   d = (t_hi - y_hi) + (t_lo - y_lo): the hi difference is exact for close
//   points (Sterbenz) and the lo parts restore the bits lost in rounding.
// The pair loop runs on the FP32 pipe (MUFU reciprocal and log); partial sums
// are kept in two FP32 levels (blocks of 16 pairs) and combined per target in
// FP32 across lanes, then in FP64.  Exactly coincident pairs are skipped.
// L2P: FP32 Horner, FP64 final combination of psi.
constexpr int STAGE = 256;     // sources staged per warp (double-float kernel)
constexpr int STAGE32 = 192;   // FP32 kernel: smaller stage, 7 blocks of 4 warps per SM

struct Eval32Args {
    TreeView T;
    const int* leaves;
    int64_t n_leaves;
    const int64_t* d_n_leaves;      // graph mode: the leaf count on the device (n_leaves: the capacity)
    const float4* soff;       // [2N]: (hi offset, q), (lo offset, 0) of each source from its leaf centre
    const float4* toff;       // [2M]: (hi, x.z), (lo, 0) offset of each sorted target from its leaf centre
    const float4* dc;         // [2 n_p2p]: (hi, 0), (lo, 0) offset of each near leaf's centre from the target leaf's
    const double4_32a* tgt;
    const uint32_t* tperm;
    const int64_t* p2p_off;
    const uint32_t* p2p_src;
    const float* local;       // FP32 local expansions (FP32 far field)
    const float* base_mpole;
    const dflt* local_df;     // double-float local expansions (double-float far field)
    const dflt* base_mpole_df;
    int p;
    int want_psi;
    int zero_mean;
    double* psi;
    double* alpha;
    unsigned long long* leaf_ctr;   // zero at launch: the warps take target leaves from it one at a time
    // double-float far field: the near field's sums per sorted target, for k_finish_dfar:
    // nf[2t] = (x.h, x.l, y.h, y.l), nf[2t + 1] = (z.h, z.l, sum q, sum q log2 d^2), and its leaf
    float4* nf;
    int* tleaf;
    const FrameDF* frames;    // the nodes' double-float frames (k_frame_df)
    int64_t M;                // sorted targets
};

__device__ __forceinline__ float group_sumf(float v, int lpt)
{
    for (int o = lpt >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// error-free a + b = s + e (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float* s, float* e)
{
    const float x = a + b;
    const float bb = x - a;
    *e = (a - (x - bb)) + (b - bb);
    *s = x;
}

// The staged near sources of one warp, packed by pairs of sources (a, b) =
// (2P, 2P+1) and negated, so that one 16-byte load yields (x_a, x_b, y_a, y_b)
// and the pair loop runs on packed FP32x2 instructions: hi offsets (x, y), (z,
// mass), lo offsets (x, y), (z, unused), all from the target leaf's centre.
// Every array has a 16-byte stride, so that the four loads of pair P (and the
// stores of the staging) share one address with fixed displacements.
struct Stage32 {
    float4 hxy[STAGE32 / 2];
    float4 hzq[STAGE32 / 2];
    float4 lxy[STAGE32 / 2];
    float4 lz[STAGE32 / 2];
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// base-2 logarithm, approximate, subnormal input flushed to zero: the pair
// loop's d^2 is either at least FLT_MIN or the pair is treated as coincident
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Near-field sums of one target over the staged source pairs P = sub, sub + lpt,
// ...: blocks of (up to) 16 pairs per lane in packed FP32 (the two halves sum
// the even and the odd sources), then the outer FP32 level acc.  The logarithm
// is accumulated in base 2 (acc[4] = sum q log2 d^2).  1/d^2 is the
// approximate reciprocal (as in __fdividef).  The mass sum acc[3] is the same
// for every target of the stage: it is added once per target from the stage's
// total (stage_q), less the mass of the sources a target skips.
//
// A source at the target's own position (d^2 = 0, or below FLT_MIN, where the
// flushed reciprocal and logarithm are not finite) is left out.  The masked
// block tests every pair for it and sums the mass it skips (iq); the plain
// block does not test: there 1/d^2 = inf and its x sum turns inf or NaN, so a
// plain block whose x sum is not finite is summed again masked.  When the
// targets are the sources themselves every target meets one such block; there
// (MASK) every block is masked.
template <bool PSI, bool MASKED>
__device__ __forceinline__ void pair_block32(const Stage32& S, int P0, int P1, int lpt, const float2& tx,
                                             const float2& ty, const float2& tz, const float2& ux, const float2& uy,
                                             const float2& uz, float2& ix, float2& iy, float2& iz, float2& iq,
                                             float2& il)
{
#pragma unroll 2
    for (int P = P0; P < P1; P += lpt) {
        const float4 a = S.hxy[P], b = S.hzq[P], c = S.lxy[P], d = S.lz[P];
        const float2 dx = __fadd2_rn(__fadd2_rn(tx, f2(a.x, a.y)), __fadd2_rn(ux, f2(c.x, c.y)));
        const float2 dy = __fadd2_rn(__fadd2_rn(ty, f2(a.z, a.w)), __fadd2_rn(uy, f2(c.z, c.w)));
        const float2 dz = __fadd2_rn(__fadd2_rn(tz, f2(b.x, b.y)), __fadd2_rn(uz, f2(d.x, d.y)));
        const float2 d2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        float2 q = f2(b.z, b.w);
        float2 den = d2;
        if (MASKED) {
            const bool oka = d2.x >= FLT_MIN_F, okb = d2.y >= FLT_MIN_F;
            iq = __fadd2_rn(iq, f2(oka ? 0.f : q.x, okb ? 0.f : q.y));     // the mass skipped
            q = f2(oka ? q.x : 0.f, okb ? q.y : 0.f);
            den = f2(oka ? d2.x : 1.f, okb ? d2.y : 1.f);
        }
        const float2 wq = __fmul2_rn(q, f2(rcp_approx(den.x), rcp_approx(den.y)));
        ix = __ffma2_rn(wq, dx, ix);
        iy = __ffma2_rn(wq, dy, iy);
        iz = __ffma2_rn(wq, dz, iz);
        if (PSI) il = __ffma2_rn(q, f2(lg2_approx(den.x), lg2_approx(den.y)), il);
    }
}

// COMP: the outer level of the three alpha sums is compensated (two-sum of
// each block's sum into acc, the rounding errors collected in accl), for the
// path whose far field is carried in double-float.
template <bool PSI, bool MASK, bool COMP>
__device__ __forceinline__ void pair_sums32(const Stage32& S, int npair, int sub, int lpt, const float4& th,
                                            const float4& tl, float stage_q, float* acc, float* accl)
{
    const float2 tx = f2(th.x, th.x), ty = f2(th.y, th.y), tz = f2(th.z, th.z);
    const float2 ux = f2(tl.x, tl.x), uy = f2(tl.y, tl.y), uz = f2(tl.z, tl.z);
    if (sub == 0) acc[3] += stage_q;          // once per target (its lanes' sums are added up)
    for (int P = sub; P < npair;) {
        const int pend = min(npair, P + 16 * lpt);
        float2 ix = f2(0.f, 0.f), iy = ix, iz = ix, iq = ix, il = ix;   // inner FP32 level
        pair_block32<PSI, MASK>(S, P, pend, lpt, tx, ty, tz, ux, uy, uz, ix, iy, iz, iq, il);
        if (!MASK && !(fabsf(ix.x) < INFINITY && fabsf(ix.y) < INFINITY)) {
            ix = f2(0.f, 0.f); iy = ix; iz = ix; iq = ix; il = ix;
            pair_block32<PSI, true>(S, P, pend, lpt, tx, ty, tz, ux, uy, uz, ix, iy, iz, iq, il);
        }
        if (COMP) {
            float e0, e1, e2;
            two_sum(acc[0], ix.x + ix.y, &acc[0], &e0);
            two_sum(acc[1], iy.x + iy.y, &acc[1], &e1);
            two_sum(acc[2], iz.x + iz.y, &acc[2], &e2);
            accl[0] += e0; accl[1] += e1; accl[2] += e2;
        } else {
            acc[0] += ix.x + ix.y; acc[1] += iy.x + iy.y; acc[2] += iz.x + iz.y;
        }
        acc[3] -= iq.x + iq.y; acc[4] += il.x + il.y;
        P = pend;
    }
}

// L2P in the leaf frame (FP32 Horner, FP64 final psi) plus the near-field sums
// acc, written for sorted target tix.
// A leaf's frame in FP32, formed once per leaf: e_theta, e_phi, 2 c, 1/r.
struct LeafFrame32 {
    float et[3], ep[3], c2[3], inv_r;
};

template <bool PSI>
__device__ __forceinline__ void finish_target32(const Eval32Args& A, const LeafFrame32& G, const float* L,
                                                size_t tix, const float4& th, const float4& tl, const float* acc,
                                                double shift)
{
    const float ox = acc[0], oy = acc[1], oz = acc[2], oq = acc[3], ol = acc[4];
    const float tx = th.x + tl.x, ty = th.y + tl.y, tz = th.z + tl.z;
    const float D2 = tx * tx + ty * ty + tz * tz;
    const float den = 2.f - 0.5f * D2;
    const float wu = (tx * G.et[0] + ty * G.et[1] + tz * G.et[2]) / den;
    const float wv = (tx * G.ep[0] + ty * G.ep[1] + tz * G.ep[2]) / den;
    const float inv_r = G.inv_r;
    const float omx = wu * inv_r, omy = wv * inv_r;
    float frx = 0.f, fry = 0.f, fdx = 0.f, fdy = 0.f;
    for (int l = A.p; l >= 1; --l) {
        const float ax = L[2 * l], ay = L[2 * l + 1];
        const float nfx = frx * omx - fry * omy + ax;
        const float nfy = frx * omy + fry * omx + ay;
        const float ndx = fdx * omx - fdy * omy + ax * (float)l;
        const float ndy = fdx * omy + fdy * omx + ay * (float)l;
        frx = nfx; fry = nfy; fdx = ndx; fdy = ndy;
    }
    const float Fx = frx * omx - fry * omy;
    const float Fpx = fdx * inv_r, Fpy = fdy * inv_r;
    const float Qf = L[1];
    const float w2 = wu * wu + wv * wv;
    const float au = (1.f + w2) * Fpx - Qf * wu;
    const float av = -(1.f + w2) * Fpy - Qf * wv;
    // c + x = 2c + (x - c); x itself to FP32 accuracy as c + (x - c)
    const float cxx = G.c2[0] + tx, cyy = G.c2[1] + ty, czz = G.c2[2] + tz;
    const float xx = 0.5f * G.c2[0] + tx, xy = 0.5f * G.c2[1] + ty, xz = 0.5f * G.c2[2] + tz;
    float a3x = au * (G.et[0] - wu * cxx) + av * (G.ep[0] - wv * cxx);
    float a3y = au * (G.et[1] - wu * cyy) + av * (G.ep[1] - wv * cyy);
    float a3z = au * (G.et[2] - wu * czz) + av * (G.ep[2] - wv * czz);
    const float i2p = (float)INV2PI;
    a3x += i2p * (ox - 0.5f * xx * oq);
    a3y += i2p * (oy - 0.5f * xy * oq);
    a3z += i2p * (oz - 0.5f * xz * oq);
    const float rho = sqrtf(xx * xx + xy * xy);
    float cp = 1.f, sp = 0.f;
    if (rho > 0.f) { cp = xx / rho; sp = xy / rho; }
    const uint32_t o = A.tperm[tix];
    if (A.alpha) {
        A.alpha[2 * (size_t)o] = (double)(a3x * (xz * cp) + a3y * (xz * sp) - a3z * rho);
        A.alpha[2 * (size_t)o + 1] = (double)(-a3x * sp + a3y * cp);
    }
    if (PSI) {
        const double psi_e = (double)L[0] + (double)L[1] * (LOG2 + (double)log1pf(-0.25f * D2)) + 2.0 * (double)Fx;
        A.psi[o] = psi_e + INV4PI * (LOG2 * (double)ol - LOG4 * (double)oq) + shift;
    }
}

// Far field in double-float (the 1e-6 path).  The far field at a target and
// the near field of its direct-act leaves are both large next to their sum
// wherever the mass is spread smoothly (the near leaves' field and the field
// of the hole they leave in the far mass nearly cancel), so both are formed
// and combined in double-float before the result is rounded.  L2P: w from
// the (hi, lo) target offset and the leaf frame in double-float, F'(w) by a
// double-float Horner recurrence, alpha on the chart's unit vectors
// e_u = e_theta(L) - u (c + x), e_v = e_phi(L) - v (c + x), where the near
// field's sums are projected (their radial part, x sum q / 2, projects to
// zero and is left out), then one FP32 rotation onto (e_theta, e_phi) at the
// target.  psi: F(w) by an FP32 Horner recurrence, the final sum in FP64.
struct LeafFrameDF {
    dflt et[3], ep[3], inv_r;   // e_theta, e_phi of the leaf frame and 1/r, rounded from FP64
    float c2[3];                // 2 c
};

// a / b for a double-float a and an FP32 b with ib = 1/b: the leading quotient
// and one correction from the exact remainder
__device__ __forceinline__ dflt dfl_div_f(dflt a, float b, float ib)
{
    const float q1 = __fmul_rn(a.h, ib);
    const float r = __fadd_rn(__fmaf_rn(-q1, b, a.h), a.l);
    return dfl_fast_two_sum(q1, __fmul_rn(r, ib));
}

template <bool PSI>
__device__ __forceinline__ void finish_target_dfar(const Eval32Args& A, const LeafFrameDF& G, const dflt* L,
                                                   size_t tix, const float4& th, const float4& tl, const dflt* nf,
                                                   float oq, float ol, double shift)
{
    const dflt tx(th.x, tl.x), ty(th.y, tl.y), tz(th.z, tl.z);
    const float D2 = th.x * th.x + th.y * th.y + th.z * th.z;
    const float den = 2.f - 0.5f * D2;                     // 1 + x.c
    const float iden = 1.f / den;
    const dflt wu = dfl_div_f(tx * G.et[0] + ty * G.et[1] + tz * G.et[2], den, iden);
    const dflt wv = dfl_div_f(tx * G.ep[0] + ty * G.ep[1] + tz * G.ep[2], den, iden);
    const dflt ox = wu * G.inv_r, oy = wv * G.inv_r;
    const float oxf = ox.h, oyf = oy.h;
    dflt hx(0.f, 0.f), hy(0.f, 0.f);
    float frx = 0.f, fry = 0.f;
    for (int l = A.p; l >= 1; --l) {
        const dflt cr = L[2 * l], ci = L[2 * l + 1];
        const dflt nhx = hx * ox - hy * oy + cr * (float)l;
        const dflt nhy = hx * oy + hy * ox + ci * (float)l;
        hx = nhx;
        hy = nhy;
        if (PSI) {
            const float nfx = frx * oxf - fry * oyf + cr.h;
            const float nfy = frx * oyf + fry * oxf + ci.h;
            frx = nfx;
            fry = nfy;
        }
    }
    const dflt Fpx = hx * G.inv_r, Fpy = hy * G.inv_r;    // F'(w)
    const dflt opw = dfl_two_sum(1.f, wu.h * wu.h + wv.h * wv.h);
    const dflt Q = L[1];
    const dflt au = opw * Fpx - Q * wu;
    const dflt av = -(opw * Fpy) - Q * wv;
    // the chart's unit vectors at the target (c + x = 2c + t)
    const float cxx = G.c2[0] + th.x, cyy = G.c2[1] + th.y, czz = G.c2[2] + th.z;
    const dflt eux = G.et[0] - dflt(wu.h * cxx), euy = G.et[1] - dflt(wu.h * cyy), euz = G.et[2] - dflt(wu.h * czz);
    const dflt evx = G.ep[0] - dflt(wv.h * cxx), evy = G.ep[1] - dflt(wv.h * cyy), evz = G.ep[2] - dflt(wv.h * czz);
    const dflt i2p(INV2PI);
    const dflt su = au + i2p * (nf[0] * eux + nf[1] * euy + nf[2] * euz);
    const dflt sv = av + i2p * (nf[0] * evx + nf[1] * evy + nf[2] * evz);
    const float alu = su.h + su.l, alv = sv.h + sv.l;
    // rotate onto (e_theta, e_phi) at the target x = c + t
    const float xx = 0.5f * G.c2[0] + th.x, xy = 0.5f * G.c2[1] + th.y, xz = 0.5f * G.c2[2] + th.z;
    const float rho = sqrtf(xx * xx + xy * xy);
    float cp = 1.f, sp = 0.f;
    if (rho > 0.f) { cp = xx / rho; sp = xy / rho; }
    const float etx = xz * cp, ety = xz * sp, etz = -rho;
    const float c11 = eux.h * etx + euy.h * ety + euz.h * etz, c12 = -eux.h * sp + euy.h * cp;
    const float c21 = evx.h * etx + evy.h * ety + evz.h * etz, c22 = -evx.h * sp + evy.h * cp;
    const uint32_t o = A.tperm[tix];
    if (A.alpha) {
        A.alpha[2 * (size_t)o] = (double)(alu * c11 + alv * c21);
        A.alpha[2 * (size_t)o + 1] = (double)(alu * c12 + alv * c22);
    }
    if (PSI) {
        // in double-float (this GPU's FP64 pipe runs at 1/64 of the FP32 rate), one FP64 add at the end
        const float Fx = frx * oxf - fry * oyf;
        const dflt ln2(LN2_H, LN2_L);
        const dflt psi_e = L[0] + Q * (ln2 + dflt(log1pf(-0.25f * D2))) + dflt(Fx) * 2.f;
        const dflt near = (dflt(ol) * ln2 - dflt(oq) * (ln2 * 2.f)) * dflt(INV4PI_H, INV4PI_L);
        A.psi[o] = (double)(psi_e + near) + shift;
    }
}

// The double-float finish of the 1e-6 path, one thread per sorted target: its
// leaf's frame (the node's double-float frame, 1/r, 2c), the leaf's local
// expansion and the near field's sums written by k_eval32, then
// finish_target_dfar.  Every lane works (the pair kernel's groups of 1 to 32
// targets would leave most lanes idle in this long arithmetic).
template <bool PSI>
__global__ void __launch_bounds__(128) k_finish_dfar(Eval32Args A)
{
    __shared__ double s_shift;
    if (threadIdx.x == 0) {
        double sh = 0.0;
        if (A.zero_mean)
            for (int b = 0; b < 12; ++b) sh += (double)A.base_mpole_df[(size_t)b * EXP_STRIDE + 1];
        s_shift = sh;
    }
    __syncthreads();
    const double shift = s_shift;
    for (int64_t tix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tix < A.M;
         tix += (int64_t)gridDim.x * blockDim.x) {
        const int leaf = A.tleaf[tix];
        const FrameDF F = A.frames[leaf];
        LeafFrameDF G;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            G.et[k] = F.et[k];
            G.ep[k] = F.ep[k];
            G.c2[k] = 2.f * F.c[k].h;          // (float)(2c): the scaling by 2 is exact
        }
        G.inv_r = dflt(1.f, 0.f) / F.r;
        const float4 a = A.nf[2 * tix], b = A.nf[2 * tix + 1];
        const dflt nf[3] = {dflt(a.x, a.y), dflt(a.z, a.w), dflt(b.x, b.y)};
        const float4 th = A.toff[2 * tix], tl = A.toff[2 * tix + 1];
        finish_target_dfar<PSI>(A, G, A.local_df + (size_t)leaf * EXP_STRIDE, (size_t)tix, th, tl, nf, b.z, b.w,
                                shift);
    }
}

__device__ __forceinline__ dflt group_sum_df(dflt v, int lpt)
{
    for (int o = lpt >> 1; o > 0; o >>= 1) v = v + dfl_shfl_xor(v, o);
    return v;
}

// One warp per target leaf.  The FP32 pair loop is cheap next to staging the
// sources, so each pass over the near sources serves two groups of targets at
// once: group a takes the largest power of two <= the targets left (at most
// 32), group b the power of two >= what a leaves (at most 32), e.g. 18 = 16 + 2
// and 40 = 32 + 8; each target of a group gets 32/size lanes.
// DFAR: the far field (local expansions, L2P) in double-float and the outer
// level of the near field's alpha sums compensated (finish_target_dfar).
template <bool PSI, bool MASK, bool DFAR>
__global__ void __launch_bounds__(128, 7) k_eval32(Eval32Args A)
{
    __shared__ Stage32 s_stage[4];
    __shared__ float4 s_dch[4][32], s_dcl[4][32];   // near leaves' centre offsets: hi, lo
    __shared__ int s_pre[4][33];
    __shared__ int s_first[4][32];
    __shared__ LeafFrame32 s_frame[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double shift = 0.0;
    if (A.zero_mean && !DFAR)
        for (int b = 0; b < 12; ++b) shift += (double)A.base_mpole[(size_t)b * EXP_STRIDE + 1];
    Stage32& S = s_stage[wid];
    int* pre = s_pre[wid];
    int* fst = s_first[wid];
    for (;;) {
        const int64_t w = next_leaf(A.leaf_ctr, lane);
        if (w >= dcount(A.d_n_leaves, A.n_leaves)) break;
        const int leaf = A.leaves[w];
        const int tf = A.T.tfirst[leaf], tc = A.T.tcount[leaf];
        const double* g = A.T.geom + (size_t)leaf * GEOM_STRIDE;
        const float* L = A.local + (size_t)leaf * EXP_STRIDE;
        // the leaf frame in FP32, once per leaf, kept in shared memory (the double-float far
        // field is finished by k_finish_dfar)
        LeafFrame32& G = s_frame[wid];
        __syncwarp();
        if (!DFAR) {
            if (lane < 3) {
                G.et[lane] = (float)g[3 + lane];
                G.ep[lane] = (float)g[6 + lane];
                G.c2[lane] = (float)(2.0 * g[lane]);
            }
            if (lane == 3) G.inv_r = 1.f / (float)g[10];
        }
        __syncwarp();
        const int64_t nb0 = A.p2p_off[leaf], nb1 = A.p2p_off[leaf + 1];
        for (int tb = 0; tb < tc;) {
            const int rem = tc - tb;
            const int na = min(32, 1 << (31 - __clz(rem)));
            const int rb = rem - na;
            const int nb = rb <= 0 ? 0 : min(32, 1 << (32 - __clz(rb - 1)));   // power of two >= rb
            const int lpa = 32 / na, sa = lane % lpa;
            const int lpb = nb ? 32 / nb : 32, sb = lane % lpb;
            const size_t ta = (size_t)tf + tb + lane / lpa;
            const int ib = tb + na + lane / lpb;
            const bool act_b = nb > 0 && ib < tc;
            const size_t tbx = (size_t)tf + (act_b ? ib : tb);
            const float4 tha = A.toff[2 * ta], tla = A.toff[2 * ta + 1];
            const float4 thb = A.toff[2 * tbx], tlb = A.toff[2 * tbx + 1];
            float acc_a[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, acc_b[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float accl_a[3] = {0.f, 0.f, 0.f}, accl_b[3] = {0.f, 0.f, 0.f};
            int64_t kn = nb0;
            int jn = 0;                // sources of near leaf kn already done
            while (kn < nb1) {
                // ---- records of the next (up to) 32 near leaves, one per lane
                __syncwarp();
                const int64_t k = kn + lane;
                int cnt = 0, first = 0;
                float4 rh = make_float4(0.f, 0.f, 0.f, 0.f), rl = rh;
                if (k < nb1) {
                    rh = A.dc[2 * k];
                    rl = A.dc[2 * k + 1];
                    first = __float_as_int(rh.w) + (lane == 0 ? jn : 0);
                    cnt = __float_as_int(rl.w) - (lane == 0 ? jn : 0);
                }
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += t;
                }
                const unsigned fit = __ballot_sync(FULL, k < nb1 && inc <= STAGE32);
                const int nfit = __popc(fit);
                int ns, nl;
                if (nfit == 0) { ns = STAGE32; nl = 1; }        // one leaf larger than the stage: a chunk of it
                else { ns = __shfl_sync(FULL, inc, nfit - 1); nl = nfit; }
                pre[lane] = inc - cnt;
                fst[lane] = first;
                s_dch[wid][lane] = rh;
                s_dcl[wid][lane] = rl;
                __syncwarp();
                // ---- flattened staging: position idx belongs to the largest leaf i < nl with
                // pre[i] <= idx, found by stepping on from the previous position's leaf; its
                // offset is moved from its leaf's centre to the target leaf's (two-sum with the
                // near leaf's centre offset) and stored negated in the pair-packed stage
                float sq = 0.f;        // mass staged by this lane
                for (int idx = lane, lo = 0; idx < ns; idx += 32) {
                    while (lo + 1 < nl && pre[lo + 1] <= idx) ++lo;
                    const size_t j = (size_t)(fst[lo] + (idx - pre[lo]));
                    const float4 h = A.soff[2 * j];
                    const float4 l = A.soff[2 * j + 1];
                    const float4 dh = s_dch[wid][lo], dl = s_dcl[wid][lo];
                    // the negated offset, -(y + d) = (-y) + (-d): the same two-sum, negated exactly
                    float sx, ex_, sy, ey_, sz, ez_;
                    two_sum(-h.x, -dh.x, &sx, &ex_);
                    two_sum(-h.y, -dh.y, &sy, &ey_);
                    two_sum(-h.z, -dh.z, &sz, &ez_);
                    const int P = idx >> 1, c = idx & 1;
                    float* pa = reinterpret_cast<float*>(&S.hxy[P]);
                    float* pb = reinterpret_cast<float*>(&S.hzq[P]);
                    float* pc = reinterpret_cast<float*>(&S.lxy[P]);
                    float* pd = reinterpret_cast<float*>(&S.lz[P]);
                    pa[c] = sx;
                    pa[2 + c] = sy;
                    pb[c] = sz;
                    pb[2 + c] = h.w;
                    sq += h.w;
                    pc[c] = ex_ - (l.x + dl.x);
                    pc[2 + c] = ey_ - (l.y + dl.y);
                    pd[c] = ez_ - (l.z + dl.z);
                }
                if ((ns & 1) && lane == 0) {        // an odd count: a massless partner 4 away
                    const int P = ns >> 1;
                    reinterpret_cast<float*>(&S.hxy[P])[1] = -4.f;
                    reinterpret_cast<float*>(&S.hxy[P])[3] = 0.f;
                    reinterpret_cast<float*>(&S.hzq[P])[1] = 0.f;
                    reinterpret_cast<float*>(&S.hzq[P])[3] = 0.f;
                    reinterpret_cast<float*>(&S.lxy[P])[1] = 0.f;
                    reinterpret_cast<float*>(&S.lxy[P])[3] = 0.f;
                    reinterpret_cast<float*>(&S.lz[P])[1] = 0.f;
                }
                if (nfit == 0) jn += STAGE32;
                else { kn += nfit; jn = 0; }
                __syncwarp();
                sq = group_sumf(sq, 32);
                pair_sums32<PSI, MASK, DFAR>(S, (ns + 1) >> 1, sa, lpa, tha, tla, sq, acc_a, accl_a);
                if (nb) pair_sums32<PSI, MASK, DFAR>(S, (ns + 1) >> 1, sb, lpb, thb, tlb, sq, acc_b, accl_b);
            }
            if (DFAR) {
                // the sums go to k_finish_dfar (one thread per target, every lane busy in the
                // long double-float finish): the lane that holds a target's group sums writes them
                dflt nfa[3], nfb[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    nfa[c] = group_sum_df(dfl_two_sum(acc_a[c], accl_a[c]), lpa);
                    nfb[c] = group_sum_df(dfl_two_sum(acc_b[c], accl_b[c]), lpb);
                }
#pragma unroll
                for (int c = 3; c < 5; ++c) {
                    acc_a[c] = group_sumf(acc_a[c], lpa);
                    acc_b[c] = group_sumf(acc_b[c], lpb);
                }
                if (sa == 0) {
                    A.nf[2 * ta] = make_float4(nfa[0].h, nfa[0].l, nfa[1].h, nfa[1].l);
                    A.nf[2 * ta + 1] = make_float4(nfa[2].h, nfa[2].l, acc_a[3], acc_a[4]);
                    A.tleaf[ta] = leaf;
                }
                if (act_b && sb == 0) {
                    A.nf[2 * tbx] = make_float4(nfb[0].h, nfb[0].l, nfb[1].h, nfb[1].l);
                    A.nf[2 * tbx + 1] = make_float4(nfb[2].h, nfb[2].l, acc_b[3], acc_b[4]);
                    A.tleaf[tbx] = leaf;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    acc_a[c] = group_sumf(acc_a[c], lpa);
                    acc_b[c] = group_sumf(acc_b[c], lpb);
                }
                if (sa == 0) finish_target32<PSI>(A, G, L, ta, tha, tla, acc_a, shift);
                if (act_b && sb == 0) finish_target32<PSI>(A, G, L, tbx, thb, tlb, acc_b, shift);
            }
            tb += na + nb;
        }
    }
}

// ------------------------------------------------------------------------
// Double-float evaluation (SFMM_MIXED_DF, stated error 1e-10).  The same
// staging as k_eval32; the pair loop carries every quantity as an unevaluated
// sum of two FP32 numbers (about 48 significant bits), on the FP32 pipe:
//   d = t - y from the (hi, lo) offsets with an error-free two-difference,
//   d^2 with error-free products (fma), 1/d^2 from the MUFU reciprocal and one
//   Newton correction, the alpha and sum-q accumulators as FP32 pairs,
//   log d^2 = e ln2 + log c_j + log1p(r): c_j = 1 + j/128 from the top mantissa
//   bits, log c_j and 1/c_j from a 128-entry table computed in FP64 on the host
//   (a table-driven logarithm in the manner of Tang, ACM TOMS 16, 1990),
//   |r| < 2^-7 so r - r^2/2 + ... + r^6/6 reaches double-float accuracy.
// L2P (double-float local expansions) and the final combination in double-float.
// a - b for double-float a = (ah, al), b = (bh, bl): two-difference of the
// leading parts, the tails added to its error, then renormalised -- for close
// points the leading parts cancel and the difference lives in the tails (the
// tails of the two offsets can then exceed the difference's own last place,
// so the renormalisation is needed before its square is formed)
__device__ __forceinline__ dflt dfl_diff(float ah, float al, float bh, float bl)
{
    const dflt s = dfl_two_sum(ah, -bh);
    return dfl_fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(al, bl)));
}

struct EvalDfArgs {
    TreeView T;
    const int* leaves;
    int64_t n_leaves;
    const int64_t* d_n_leaves;      // graph mode: the leaf count on the device (n_leaves: the capacity)
    const float4* soff;
    const float4* toff;
    const float4* dc;
    const double4_32a* tgt;
    const uint32_t* tperm;
    const int64_t* p2p_off;
    const uint32_t* p2p_src;
    const dflt* local;         // double-float local expansions
    const dflt* base_mpole;
    const float4* log_tab;     // [129]: log c_j and 1/c_j as (hi, lo) pairs, then log 2
    int p;
    int zero_mean;
    double* psi;
    double* alpha;
    unsigned long long* leaf_ctr;   // zero at launch: the warps take target leaves from it one at a time
    // the adjoint (k_eval_df<PSI, true>): the sources' tangent dipoles as (hi, lo)
    // float4 pairs, the targets' weights w (the forward masses) and the output
    // w grad Phi [M][3]; psi then receives Phi
    const float4* doff;
    const void* w;
    int w_f32;
    double* grad3;
    // the forward (k_eval_df<PSI, false>) writes each sorted target's near-field sums,
    // nf[3t] = (x.h, x.l, y.h, y.l), nf[3t + 1] = (z.h, z.l, q.h, q.l), nf[3t + 2] =
    // (log.h, log.l, 0, 0), and its leaf; k_finish_df reads them with the nodes'
    // double-float frames
    float4* nf;
    int* tleaf;
    const FrameDF* frames;
    int64_t M;                // sorted targets
};

// ---- packed double-float: the two halves of every FP32x2 register pair carry
// two sources' double-float quantities (h + l), with the same operations as the
// scalar double-float helpers; a - b is fma(b, -1, a), exact like a subtraction.
struct df2 {
    float2 h, l;
};
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ df2 p_fast_two_sum(float2 a, float2 b)        // |a| >= |b| (or a == 0)
{
    const float2 s = p_add(a, b);
    return df2{s, p_sub(b, p_sub(s, a))};
}
// (t - y) for double-float t, y: the two-difference of the leading parts, the
// tails added to its error, renormalised (as dfl_diff)
__device__ __forceinline__ df2 p_diff(float2 th, float2 tl, float2 yh, float2 yl)
{
    const float2 s = p_sub(th, yh);
    const float2 bb = p_sub(s, th);
    const float2 e = p_sub(p_sub(th, p_sub(s, bb)), p_add(yh, bb));     // (th - (s - bb)) + (-yh - bb)
    return p_fast_two_sum(s, p_add(e, p_sub(tl, yl)));
}
__device__ __forceinline__ df2 p_two_sum(float2 a, float2 b)
{
    const float2 s = p_add(a, b);
    const float2 bb = p_sub(s, a);
    return df2{s, p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb))};
}
// acc += a * b, acc left unnormalised (as dfl_mac)
__device__ __forceinline__ void p_mac(df2& acc, const df2& a, const df2& b)
{
    const float2 pr = p_mul(a.h, b.h);
    const float2 e = p_fma(a.h, b.l, p_fma(a.l, b.h, p_fma(a.h, b.h, p_neg(pr))));
    const df2 s = p_two_sum(acc.h, pr);
    acc.h = s.h;
    acc.l = p_add(acc.l, p_add(s.l, e));
}
__device__ __forceinline__ df2 p_mul_lazy(const df2& a, const df2& b)
{
    const float2 pr = p_mul(a.h, b.h);
    return df2{pr, p_fma(a.h, b.l, p_fma(a.l, b.h, p_fma(a.h, b.h, p_neg(pr))))};
}
__device__ __forceinline__ df2 p_mul(const df2& a, const df2& b)
{
    const float2 pr = p_mul(a.h, b.h);
    const float2 e = p_fma(a.h, b.h, p_neg(pr));
    return p_fast_two_sum(pr, p_fma(a.h, b.l, p_fma(a.l, b.h, e)));
}
__device__ __forceinline__ dflt p_lo_half(const df2& a) { return dflt(a.h.x, a.l.x); }
__device__ __forceinline__ dflt p_hi_half(const df2& a) { return dflt(a.h.y, a.l.y); }

// The forward double-float stage of one warp, packed by pairs of sources (a, b) =
// (2P, 2P + 1): xy[P] = (x_a, x_b, y_a, y_b), zq[P] = (z_a, z_b, q_a, q_b), leading
// parts (h) and tails (l), the offsets from the target leaf's centre.  It fills
// the same shared memory as the per-source stage of the adjoint.
struct StageDF {
    const float4* hxy;
    const float4* hzq;
    const float4* lxy;
    const float4* lzq;
};

// Near-field sums of one target in double-float over the packed stage: np pairs
// P = sub, sub + lpt, ... (ptail: the pair whose second source is the massless
// partner of an odd count, or -1), in blocks of up to 16 pairs (32 sources) per
// lane; the packed sums are added to acc = (x, y, z sums of q d / d^2, sum q log
// d^2, the mass skipped at coincident points) at the end.  EQM (every staged
// source has the same mass qm): sum q log d^2 = qm log prod d^2, so per block the
// lane multiplies the d^2 (their mantissas, in double-float, the exponents summed
// as an integer) and takes one logarithm per block.
template <bool PSI, bool EQM>
__device__ __forceinline__ void pair_sums_df2(const StageDF& S, int np, int ptail, int sub, int lpt, const float4& th,
                                              const float4& tl, dflt qm, const float4* __restrict__ tab, dflt* acc)
{
    const float2 txh = f2(th.x, th.x), tyh = f2(th.y, th.y), tzh = f2(th.z, th.z);
    const float2 txl = f2(tl.x, tl.x), tyl = f2(tl.y, tl.y), tzl = f2(tl.z, tl.z);
    const float2 z2 = f2(0.f, 0.f);
    df2 ax{z2, z2}, ay{z2, z2}, az{z2, z2}, al{z2, z2};
    dflt skip(0.f, 0.f);
    for (int P0 = sub; P0 < np; P0 += 16 * lpt) {
        const int P1 = min(np, P0 + 16 * lpt);
        df2 prod{f2(1.f, 1.f), z2};
        int ecnt = 0;
        for (int P = P0; P < P1; P += lpt) {
            const float4 A = S.hxy[P], B = S.hzq[P], C = S.lxy[P], D = S.lzq[P];
            const df2 dx = p_diff(txh, txl, f2(A.x, A.y), f2(C.x, C.y));
            const df2 dy = p_diff(tyh, tyl, f2(A.z, A.w), f2(C.z, C.w));
            const df2 dz = p_diff(tzh, tzl, f2(B.x, B.y), f2(D.x, D.y));
            // d^2: exact squares of the leading parts, two exact two-sums
            const float2 px = p_mul(dx.h, dx.h), py = p_mul(dy.h, dy.h), pz = p_mul(dz.h, dz.h);
            const float2 ex2 = p_fma(p_add(dx.h, dx.h), dx.l, p_fma(dx.h, dx.h, p_neg(px)));
            const float2 ey2 = p_fma(p_add(dy.h, dy.h), dy.l, p_fma(dy.h, dy.h, p_neg(py)));
            const float2 ez2 = p_fma(p_add(dz.h, dz.h), dz.l, p_fma(dz.h, dz.h, p_neg(pz)));
            const df2 s1 = p_two_sum(px, py);
            const df2 s2 = p_two_sum(s1.h, pz);
            df2 d2 = p_fast_two_sum(s2.h, p_add(p_add(s1.l, s2.l), p_add(p_add(ex2, ey2), ez2)));
            df2 q{f2(B.z, B.w), f2(D.z, D.w)};
            // coincident pairs (d^2 below the normal range) contribute nothing; their mass is skipped
            const bool oka = d2.h.x >= FLT_MIN_F, okb = d2.h.y >= FLT_MIN_F;
            if (!(oka && okb)) {
                if (!oka) {
                    skip = skip + dflt(q.h.x, q.l.x);
                    q.h.x = 0.f; q.l.x = 0.f; d2.h.x = 1.f; d2.l.x = 0.f;
                }
                if (!okb) {
                    skip = skip + dflt(q.h.y, q.l.y);
                    q.h.y = 0.f; q.l.y = 0.f; d2.h.y = 1.f; d2.l.y = 0.f;
                }
            }
            // 1/d^2: MUFU reciprocal and one Newton step
            const float2 r0 = f2(rcp_approx(d2.h.x), rcp_approx(d2.h.y));
            const float2 e0 = p_fma(p_neg(d2.l), r0, p_fma(p_neg(d2.h), r0, f2(1.f, 1.f)));
            const df2 wq = p_mul_lazy(df2{r0, p_mul(r0, e0)}, q);
            p_mac(ax, wq, dx);
            p_mac(ay, wq, dy);
            p_mac(az, wq, dz);
            if (PSI) {
                if (EQM) {
                    // d^2 = m 2^k, m in [1, 2): multiply the mantissas, sum the exponents; the
                    // massless partner of an odd count multiplies by 1
                    const int ba = __float_as_int(d2.h.x) >> 23, bb = __float_as_int(d2.h.y) >> 23;
                    const float2 sc = f2(__int_as_float((254 - ba) << 23), __int_as_float((254 - bb) << 23));
                    df2 m{p_mul(d2.h, sc), p_mul(d2.l, sc)};
                    int kb = bb - 127;
                    if (P == ptail) {
                        m.h.y = 1.f; m.l.y = 0.f; kb = 0;
                    }
                    prod = p_mul(prod, m);
                    ecnt += (ba - 127) + kb;
                } else {
                    const dflt la = dfl_log_lazy(dflt(d2.h.x, d2.l.x), tab), lb = dfl_log_lazy(dflt(d2.h.y, d2.l.y), tab);
                    p_mac(al, df2{f2(la.h, lb.h), f2(la.l, lb.l)}, q);
                }
            }
        }
        if (PSI && EQM) {
            // log of the product of both halves + ecnt log 2 (ecnt exact in FP32)
            const dflt pr = p_lo_half(prod) * p_hi_half(prod);
            const dflt lg = dfl_norm(dfl_log_lazy(pr, tab)) + dflt((float)ecnt) * dflt(LN2_H, LN2_L);
            dfl_mac(acc[3], lg, qm);
        }
    }
    acc[0] = acc[0] + dfl_norm(p_lo_half(ax)) + dfl_norm(p_hi_half(ax));
    acc[1] = acc[1] + dfl_norm(p_lo_half(ay)) + dfl_norm(p_hi_half(ay));
    acc[2] = acc[2] + dfl_norm(p_lo_half(az)) + dfl_norm(p_hi_half(az));
    if (PSI && !EQM) acc[3] = acc[3] + dfl_norm(p_lo_half(al)) + dfl_norm(p_hi_half(al));
    acc[4] = acc[4] + skip;
}

// A leaf's frame in double-float, formed once per leaf: e_theta, e_phi, the
// centre c and 1/r, rounded from FP64.
struct LeafFrameD2 {
    dflt et[3], ep[3], c[3], inv_r;
};

// L2P in the leaf frame and the combination with the near field's sums for
// sorted target tix, all in double-float (no FP64 instructions: this GPU's
// FP64 pipe runs at 1/64 of the FP32 rate).  t = x - c from the target's
// (hi, lo) offset; w = (t.e_theta + i t.e_phi) / (1 + x.c), 1 + x.c = 2 - |t|^2/2;
// F(w) and F'(w) by Horner recurrences; alpha on the chart vectors
// e_u = e_theta - u (c + x), e_v = e_phi - v (c + x) plus the near field's
// sums, rotated onto (e_theta, e_phi) at x; psi = C + Q (log 2 + log(1 - |t|^2/4))
// + 2 Re F + (sum q log d^2 - log 4 sum q) / 4pi.
template <bool PSI>
__device__ __forceinline__ void finish_target_df(const EvalDfArgs& A, const LeafFrameD2& G, const dflt* L,
                                                 size_t tix, const float4& th, const float4& tl, const dflt* nf,
                                                 const float4* __restrict__ tab, double shift)
{
    const dflt tx(th.x, tl.x), ty(th.y, tl.y), tz(th.z, tl.z);
    const dflt D2 = tx * tx + ty * ty + tz * tz;
    const dflt den = dflt(2.f, 0.f) - D2 * 0.5f;
    const dflt wu = (tx * G.et[0] + ty * G.et[1] + tz * G.et[2]) / den;
    const dflt wv = (tx * G.ep[0] + ty * G.ep[1] + tz * G.ep[2]) / den;
    const dflt ox = wu * G.inv_r, oy = wv * G.inv_r;
    dflt fx(0.f, 0.f), fy(0.f, 0.f), hx(0.f, 0.f), hy(0.f, 0.f);
    for (int l = A.p; l >= 1; --l) {
        const dflt cr = L[2 * l], ci = L[2 * l + 1];
        if (PSI) {
            const dflt nfx = fx * ox - fy * oy + cr, nfy = fx * oy + fy * ox + ci;
            fx = nfx; fy = nfy;
        }
        const dflt nhx = hx * ox - hy * oy + cr * (float)l, nhy = hx * oy + hy * ox + ci * (float)l;
        hx = nhx; hy = nhy;
    }
    const dflt Fpx = hx * G.inv_r, Fpy = hy * G.inv_r;    // F'(w)
    const dflt C = L[0], Q = L[1];
    const dflt opw = dflt(1.f, 0.f) + (wu * wu + wv * wv);
    const dflt au = opw * Fpx - Q * wu;
    const dflt av = -(opw * Fpy) - Q * wv;
    // x = c + t and c + x = 2c + t
    const dflt xx = G.c[0] + tx, xy = G.c[1] + ty, xz = G.c[2] + tz;
    const dflt cxx = G.c[0] + xx, cyy = G.c[1] + xy, czz = G.c[2] + xz;
    const dflt i2p(INV2PI);
    const dflt sx = nf[0] - xx * (nf[3] * 0.5f), sy = nf[1] - xy * (nf[3] * 0.5f), sz = nf[2] - xz * (nf[3] * 0.5f);
    const dflt a3x = au * (G.et[0] - wu * cxx) + av * (G.ep[0] - wv * cxx) + i2p * sx;
    const dflt a3y = au * (G.et[1] - wu * cyy) + av * (G.ep[1] - wv * cyy) + i2p * sy;
    const dflt a3z = au * (G.et[2] - wu * czz) + av * (G.ep[2] - wv * czz) + i2p * sz;
    // rotate onto (e_theta, e_phi) at x (phi = 0 at the poles)
    const dflt rho = dfl_sqrt(xx * xx + xy * xy);
    dflt cp(1.f, 0.f), sp(0.f, 0.f);
    if (rho.h > 0.f) { cp = xx / rho; sp = xy / rho; }
    const uint32_t o = A.tperm[tix];
    if (A.alpha) {
        A.alpha[2 * (size_t)o] = (double)(a3x * (xz * cp) + a3y * (xz * sp) - a3z * rho);
        A.alpha[2 * (size_t)o + 1] = (double)(a3y * cp - a3x * sp);
    }
    if (PSI) {
        const dflt F = fx * ox - fy * oy;                   // Re F(w)
        const dflt ln2(LN2_H, LN2_L);
        const dflt psi_e = C + Q * (ln2 + dfl_log1m(D2 * 0.25f, tab)) + F * 2.f;
        const dflt near = (nf[4] - nf[3] * (ln2 * 2.f)) * dflt(INV4PI);
        A.psi[o] = (double)(psi_e + near) + shift;
    }
}

__device__ __forceinline__ dflt group_sum_dfl(dflt v, int lpt)
{
    for (int o = lpt >> 1; o > 0; o >>= 1) v = v + dfl_shfl_xor(v, o);
    return v;
}

// The adjoint's near-field sums of one target (a forward source) over the
// staged adjoint sources (forward targets, charges h and tangent dipoles g):
// acc[0..3] as pair_sums_df2 (per source) for the charges (CHG: the stage has a
// non-zero charge), acc[4] the mass skipped at coincident points, and for the dipoles,
// with G(x, y) = (1/4pi) log |x - y|^2 + const and d = x - y:
//   acc[5] = sum (g . (y - x)) / d^2      (the potential, times 2 / 4pi)
//   acc[6..8] = sum 2 (g . d) d / d^4 - g / d^2   (its gradient in x, likewise).
template <bool PSI, bool CHG, bool EQM>
__device__ __forceinline__ void pair_sums_adj_df(const float4* __restrict__ yh, const float4* __restrict__ yl,
                                                 const float4* __restrict__ gh_, const float4* __restrict__ gl_,
                                                 int ns, int sub, int lpt, const float4& th, const float4& tl,
                                                 dflt qm, const float4* __restrict__ tab, dflt* acc)
{
    for (int j0 = sub; j0 < ns; j0 += 16 * lpt) {
        const int j1 = min(ns, j0 + 16 * lpt);
        dflt prod(1.f, 0.f);
        int ecnt = 0;
        for (int j = j0; j < j1; j += lpt) {
            const float4 h = yh[j];
            const float4 l = yl[j];
            const dflt dx = dfl_diff(th.x, tl.x, h.x, l.x);
            const dflt dy = dfl_diff(th.y, tl.y, h.y, l.y);
            const dflt dz = dfl_diff(th.z, tl.z, h.z, l.z);
            const float px = __fmul_rn(dx.h, dx.h), py = __fmul_rn(dy.h, dy.h), pz = __fmul_rn(dz.h, dz.h);
            const float ex2 = __fmaf_rn(__fadd_rn(dx.h, dx.h), dx.l, __fmaf_rn(dx.h, dx.h, -px));
            const float ey2 = __fmaf_rn(__fadd_rn(dy.h, dy.h), dy.l, __fmaf_rn(dy.h, dy.h, -py));
            const float ez2 = __fmaf_rn(__fadd_rn(dz.h, dz.h), dz.l, __fmaf_rn(dz.h, dz.h, -pz));
            const dflt s1 = dfl_two_sum(px, py);
            const dflt s2 = dfl_two_sum(s1.h, pz);
            dflt d2 = dfl_fast_two_sum(s2.h, __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(ex2, ey2), ez2)));
            const bool ok = d2.h >= FLT_MIN_F;
            dflt q = dflt(h.w, l.w);
            if (!ok) {
                acc[4] = acc[4] + q;
                q = dflt(0.f, 0.f);
                d2 = dflt(1.f, 0.f);
            }
            const float r0 = rcp_approx(d2.h);
            const float e0 = __fmaf_rn(-d2.l, r0, __fmaf_rn(-d2.h, r0, 1.f));
            const dflt inv = ok ? dfl_fast_two_sum(r0, __fmul_rn(r0, e0)) : dflt(0.f, 0.f);   // 1/d^2
            if (CHG) {
                const dflt wq = dfl_mul_lazy(inv, q);
                dfl_mac(acc[0], wq, dx);
                dfl_mac(acc[1], wq, dy);
                dfl_mac(acc[2], wq, dz);
                if (PSI) {
                    if (EQM) {
                        const int k = (__float_as_int(d2.h) >> 23) - 127;
                        const float sc = __int_as_float((127 - k) << 23);
                        prod = prod * dflt(__fmul_rn(d2.h, sc), __fmul_rn(d2.l, sc));
                        ecnt += k;
                    } else {
                        dfl_mac(acc[3], dfl_log_lazy(d2, tab), q);
                    }
                }
            }
            // dipoles
            const float4 ga = gh_[j], gb = gl_[j];
            const dflt gx(ga.x, gb.x), gy(ga.y, gb.y), gz(ga.z, gb.z);
            const dflt gd = gx * dx + gy * dy + gz * dz;          // g . d = -(g . (y - x))
            const dflt gdi = gd * inv;
            if (PSI) acc[5] = acc[5] - gdi;
            const dflt c2 = (gdi * inv) * 2.f;
            const dflt ninv = -inv;
            dfl_mac(acc[6], c2, dx);
            dfl_mac(acc[6], ninv, gx);
            dfl_mac(acc[7], c2, dy);
            dfl_mac(acc[7], ninv, gy);
            dfl_mac(acc[8], c2, dz);
            dfl_mac(acc[8], ninv, gz);
        }
        if (CHG && PSI && EQM) {
            const dflt lg = dfl_norm(dfl_log_lazy(prod, tab)) + dflt((float)ecnt) * dflt(LN2_H, LN2_L);
            dfl_mac(acc[3], lg, qm);
        }
    }
}

// The adjoint's finish for target tix (a forward source): the local expansion's
// F(w) and F'(w) as in finish_target_df give Phi and its gradient; the near
// field adds the charges' sums (projected as in the forward) and the dipoles'
// gradient projected by P_x = I - x x^T; the output is w times the covariant
// gradient (a 3-vector) and Phi (+ the dipoles' potential).
template <bool PSI>
__device__ __forceinline__ void finish_target_adj_df(const EvalDfArgs& A, const LeafFrameD2& G, const dflt* L,
                                                     size_t tix, const float4& th, const float4& tl, const dflt* nf,
                                                     const float4* __restrict__ tab, double shift)
{
    const dflt tx(th.x, tl.x), ty(th.y, tl.y), tz(th.z, tl.z);
    const dflt D2 = tx * tx + ty * ty + tz * tz;
    const dflt den = dflt(2.f, 0.f) - D2 * 0.5f;
    const dflt wu = (tx * G.et[0] + ty * G.et[1] + tz * G.et[2]) / den;
    const dflt wv = (tx * G.ep[0] + ty * G.ep[1] + tz * G.ep[2]) / den;
    const dflt ox = wu * G.inv_r, oy = wv * G.inv_r;
    dflt fx(0.f, 0.f), fy(0.f, 0.f), hx(0.f, 0.f), hy(0.f, 0.f);
    for (int l = A.p; l >= 1; --l) {
        const dflt cr = L[2 * l], ci = L[2 * l + 1];
        if (PSI) {
            const dflt nfx = fx * ox - fy * oy + cr, nfy = fx * oy + fy * ox + ci;
            fx = nfx; fy = nfy;
        }
        const dflt nhx = hx * ox - hy * oy + cr * (float)l, nhy = hx * oy + hy * ox + ci * (float)l;
        hx = nhx; hy = nhy;
    }
    const dflt Fpx = hx * G.inv_r, Fpy = hy * G.inv_r;
    const dflt C = L[0], Q = L[1];
    const dflt opw = dflt(1.f, 0.f) + (wu * wu + wv * wv);
    const dflt au = opw * Fpx - Q * wu;
    const dflt av = -(opw * Fpy) - Q * wv;
    const dflt xx = G.c[0] + tx, xy = G.c[1] + ty, xz = G.c[2] + tz;
    const dflt cxx = G.c[0] + xx, cyy = G.c[1] + xy, czz = G.c[2] + xz;
    const dflt i2p(INV2PI);
    const dflt xv = xx * nf[6] + xy * nf[7] + xz * nf[8];
    const dflt hq = nf[3] * 0.5f;
    const dflt sx = nf[0] - xx * hq + nf[6] - xv * xx;
    const dflt sy = nf[1] - xy * hq + nf[7] - xv * xy;
    const dflt sz = nf[2] - xz * hq + nf[8] - xv * xz;
    const dflt a3x = au * (G.et[0] - wu * cxx) + av * (G.ep[0] - wv * cxx) + i2p * sx;
    const dflt a3y = au * (G.et[1] - wu * cyy) + av * (G.ep[1] - wv * cyy) + i2p * sy;
    const dflt a3z = au * (G.et[2] - wu * czz) + av * (G.ep[2] - wv * czz) + i2p * sz;
    const uint32_t o = A.tperm[tix];
    if (A.grad3) {
        const double wt = A.w_f32 ? (double)static_cast<const float*>(A.w)[o] : static_cast<const double*>(A.w)[o];
        A.grad3[3 * (size_t)o] = wt * (double)a3x;
        A.grad3[3 * (size_t)o + 1] = wt * (double)a3y;
        A.grad3[3 * (size_t)o + 2] = wt * (double)a3z;
    }
    if (PSI) {
        const dflt F = fx * ox - fy * oy;
        const dflt ln2(LN2_H, LN2_L);
        const dflt psi_e = C + Q * (ln2 + dfl_log1m(D2 * 0.25f, tab)) + F * 2.f;
        const dflt near = (nf[4] - nf[3] * (ln2 * 2.f)) * dflt(INV4PI) + nf[5] * i2p;
        A.psi[o] = (double)(psi_e + near) + shift;
    }
}

// One warp per target leaf; each pass over the near sources serves two groups
// of targets, as in k_eval32 (group a: the largest power of two <= the targets
// left, group b: the power of two >= what a leaves; 32 / size lanes per target).
// ADJ: the adjoint (charges and tangent dipoles at the sources, Phi and w grad
// Phi at the targets), with a stage of half the size (the dipoles are staged too).
// One target's near-field sums (x, y, z, q, log), written for k_finish_df.
__device__ __forceinline__ void store_near_df(const EvalDfArgs& A, size_t t, int leaf, const dflt* nf)
{
    A.nf[3 * t] = make_float4(nf[0].h, nf[0].l, nf[1].h, nf[1].l);
    A.nf[3 * t + 1] = make_float4(nf[2].h, nf[2].l, nf[3].h, nf[3].l);
    A.nf[3 * t + 2] = make_float4(nf[4].h, nf[4].l, 0.f, 0.f);
    A.tleaf[t] = leaf;
}

// The double-float finish of the 1e-10 path, one thread per sorted target: its
// leaf's frame (the node's double-float frame and 1/r), the leaf's local
// expansion and the near field's sums written by k_eval_df, then
// finish_target_df.  Every lane works.
template <bool PSI>
__global__ void __launch_bounds__(128) k_finish_df(EvalDfArgs A)
{
    __shared__ float4 s_tab[129];
    __shared__ double s_shift;
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = A.log_tab[i];
    if (threadIdx.x == 0) {
        double sh = 0.0;
        if (A.zero_mean)
            for (int b = 0; b < 12; ++b) sh += (double)A.base_mpole[(size_t)b * EXP_STRIDE + 1];
        s_shift = sh;
    }
    __syncthreads();
    const double shift = s_shift;
    for (int64_t tix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tix < A.M;
         tix += (int64_t)gridDim.x * blockDim.x) {
        const int leaf = A.tleaf[tix];
        const FrameDF F = A.frames[leaf];
        LeafFrameD2 G;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            G.et[k] = F.et[k];
            G.ep[k] = F.ep[k];
            G.c[k] = F.c[k];
        }
        G.inv_r = dflt(1.f, 0.f) / F.r;
        const float4 a = A.nf[3 * tix], b = A.nf[3 * tix + 1], c = A.nf[3 * tix + 2];
        const dflt nf[5] = {dflt(a.x, a.y), dflt(a.z, a.w), dflt(b.x, b.y), dflt(b.z, b.w), dflt(c.x, c.y)};
        const float4 th = A.toff[2 * tix], tl = A.toff[2 * tix + 1];
        finish_target_df<PSI>(A, G, A.local + (size_t)leaf * EXP_STRIDE, (size_t)tix, th, tl, nf, s_tab, shift);
    }
}

// 5 CTAs of 4 warps per SM for the forward (96 registers; its packed loop
// spills 72 bytes there and still runs faster than at 4), 4 for the adjoint (128
// registers without spills; at 5 it spills and ran 13 % slower)
template <bool PSI, bool ADJ>
__global__ void __launch_bounds__(128, ADJ ? 4 : 5) k_eval_df(EvalDfArgs A)
{
    constexpr int ST = ADJ ? STAGE / 2 : STAGE;
    constexpr int NACC = ADJ ? 9 : 5;
    __shared__ float4 s_hi[4][ST];
    __shared__ float4 s_lo[4][ST];
    __shared__ float4 s_gh[4][ADJ ? ST : 1];
    __shared__ float4 s_gl[4][ADJ ? ST : 1];
    __shared__ float s_dc[4][32][6];
    __shared__ int s_pre[4][33];
    __shared__ int s_first[4][32];
    __shared__ float4 s_tab[129];
    __shared__ LeafFrameD2 s_frame2[4];
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = A.log_tab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double shift = 0.0;
    if (A.zero_mean)
        for (int b = 0; b < 12; ++b) shift += (double)A.base_mpole[(size_t)b * EXP_STRIDE + 1];
    float4* yh = s_hi[wid];
    float4* yl = s_lo[wid];
    int* pre = s_pre[wid];
    int* fst = s_first[wid];
    LeafFrameD2& G = s_frame2[wid];
    for (;;) {
        const int64_t w = next_leaf(A.leaf_ctr, lane);
        if (w >= dcount(A.d_n_leaves, A.n_leaves)) break;
        const int leaf = A.leaves[w];
        const int tf = A.T.tfirst[leaf], tc = A.T.tcount[leaf];
        const double* g = A.T.geom + (size_t)leaf * GEOM_STRIDE;
        const dflt* L = A.local + (size_t)leaf * EXP_STRIDE;
        const int64_t nb0 = A.p2p_off[leaf], nb1 = A.p2p_off[leaf + 1];
        if (ADJ) {            // the adjoint finishes here; the forward in k_finish_df
            __syncwarp();
            if (lane < 3) {
                G.et[lane] = dflt(g[3 + lane]);
                G.ep[lane] = dflt(g[6 + lane]);
                G.c[lane] = dflt(g[lane]);
            }
            if (lane == 3) G.inv_r = dflt(1.0 / g[10]);
            __syncwarp();
        }
        for (int tb = 0; tb < tc;) {
            const int rem = tc - tb;
            const int na = min(32, 1 << (31 - __clz(rem)));
            const int rb = rem - na;
            const int nb = rb <= 0 ? 0 : min(32, 1 << (32 - __clz(rb - 1)));   // power of two >= rb
            const int lpa = 32 / na, sa = lane % lpa;
            const int lpb = nb ? 32 / nb : 32, sb = lane % lpb;
            const size_t ta = (size_t)tf + tb + lane / lpa;
            const int ib = tb + na + lane / lpb;
            const bool act_b = nb > 0 && ib < tc;
            const size_t tbx = (size_t)tf + (act_b ? ib : tb);
            const float4 tha = A.toff[2 * ta], tla = A.toff[2 * ta + 1];
            const float4 thb = A.toff[2 * tbx], tlb = A.toff[2 * tbx + 1];
            dflt acc_a[NACC], acc_b[NACC];
#pragma unroll
            for (int c = 0; c < NACC; ++c) acc_a[c] = acc_b[c] = dflt(0.f, 0.f);
            dflt mass(0.f, 0.f);           // the mass staged so far (the same for every target)
            int64_t kn = nb0;
            int jn = 0;
            while (kn < nb1) {
                __syncwarp();
                const int64_t k = kn + lane;
                int cnt = 0, first = 0;
                float4 rh = make_float4(0.f, 0.f, 0.f, 0.f), rl = rh;
                if (k < nb1) {
                    rh = A.dc[2 * k];
                    rl = A.dc[2 * k + 1];
                    first = __float_as_int(rh.w) + (lane == 0 ? jn : 0);
                    cnt = __float_as_int(rl.w) - (lane == 0 ? jn : 0);
                }
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += t;
                }
                const unsigned fit = __ballot_sync(FULL, k < nb1 && inc <= ST);
                const int nfit = __popc(fit);
                int ns, nl;
                if (nfit == 0) { ns = ST; nl = 1; }
                else { ns = __shfl_sync(FULL, inc, nfit - 1); nl = nfit; }
                pre[lane] = inc - cnt;
                fst[lane] = first;
                s_dc[wid][lane][0] = rh.x; s_dc[wid][lane][1] = rh.y; s_dc[wid][lane][2] = rh.z;
                s_dc[wid][lane][3] = rl.x; s_dc[wid][lane][4] = rl.y; s_dc[wid][lane][5] = rl.z;
                __syncwarp();
                // the stage's first mass: a stage whose masses all equal it takes the product logarithm
                const size_t j0 = (size_t)fst[0];
                const float q0h = A.soff[2 * j0].w, q0l = A.soff[2 * j0 + 1].w;
                bool same = true;
                dflt sq(0.f, 0.f);
                for (int idx = lane; idx < ns; idx += 32) {
                    int lo = 0, hi = nl;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (pre[mid] <= idx) lo = mid; else hi = mid;
                    }
                    const size_t j = (size_t)(fst[lo] + (idx - pre[lo]));
                    const float4 h = A.soff[2 * j];
                    const float4 l = A.soff[2 * j + 1];
                    const float* d = s_dc[wid][lo];
                    float sx, ex_, sy, ey_, sz, ez_;
                    two_sum(h.x, d[0], &sx, &ex_);
                    two_sum(h.y, d[1], &sy, &ey_);
                    two_sum(h.z, d[2], &sz, &ez_);
                    const float lx = ex_ + (l.x + d[3]), ly = ey_ + (l.y + d[4]), lz = ez_ + (l.z + d[5]);
                    if (ADJ) {
                        yh[idx] = make_float4(sx, sy, sz, h.w);
                        yl[idx] = make_float4(lx, ly, lz, l.w);
                        s_gh[wid][idx] = A.doff[2 * j];
                        s_gl[wid][idx] = A.doff[2 * j + 1];
                    } else {               // packed by pairs of sources (StageDF)
                        const int P = idx >> 1, c = idx & 1;
                        float* pa = reinterpret_cast<float*>(yh + P);
                        float* pb = reinterpret_cast<float*>(yh + ST / 2 + P);
                        float* pc = reinterpret_cast<float*>(yl + P);
                        float* pd = reinterpret_cast<float*>(yl + ST / 2 + P);
                        pa[c] = sx; pa[2 + c] = sy; pb[c] = sz; pb[2 + c] = h.w;
                        pc[c] = lx; pc[2 + c] = ly; pd[c] = lz; pd[2 + c] = l.w;
                    }
                    same = same && h.w == q0h && l.w == q0l;
                    sq = sq + dflt(h.w, l.w);
                }
                if (!ADJ && (ns & 1) && lane == 0) {    // an odd count: a massless partner 4 away
                    const int P = ns >> 1;
                    float* pa = reinterpret_cast<float*>(yh + P);
                    float* pb = reinterpret_cast<float*>(yh + ST / 2 + P);
                    float* pc = reinterpret_cast<float*>(yl + P);
                    float* pd = reinterpret_cast<float*>(yl + ST / 2 + P);
                    pa[1] = 4.f; pa[3] = 0.f; pb[1] = 0.f; pb[3] = 0.f;
                    pc[1] = 0.f; pc[3] = 0.f; pd[1] = 0.f; pd[3] = 0.f;
                }
                const bool eqm = __all_sync(FULL, same);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sq = sq + dfl_shfl_xor(sq, o);
                mass = mass + sq;
                if (nfit == 0) jn += ST;
                else { kn += nfit; jn = 0; }
                __syncwarp();
                const dflt qm(q0h, q0l);
                if (ADJ) {
                    const float4* gh = s_gh[wid];
                    const float4* gl = s_gl[wid];
                    if (eqm && q0h == 0.f && q0l == 0.f) {        // no charges in the stage: dipoles only
                        pair_sums_adj_df<PSI, false, true>(yh, yl, gh, gl, ns, sa, lpa, tha, tla, qm, s_tab, acc_a);
                        if (nb) pair_sums_adj_df<PSI, false, true>(yh, yl, gh, gl, ns, sb, lpb, thb, tlb, qm, s_tab, acc_b);
                    } else if (eqm) {
                        pair_sums_adj_df<PSI, true, true>(yh, yl, gh, gl, ns, sa, lpa, tha, tla, qm, s_tab, acc_a);
                        if (nb) pair_sums_adj_df<PSI, true, true>(yh, yl, gh, gl, ns, sb, lpb, thb, tlb, qm, s_tab, acc_b);
                    } else {
                        pair_sums_adj_df<PSI, true, false>(yh, yl, gh, gl, ns, sa, lpa, tha, tla, qm, s_tab, acc_a);
                        if (nb) pair_sums_adj_df<PSI, true, false>(yh, yl, gh, gl, ns, sb, lpb, thb, tlb, qm, s_tab, acc_b);
                    }
                } else {
                    const StageDF SD{yh, yh + ST / 2, yl, yl + ST / 2};
                    const int np = (ns + 1) >> 1, ptail = (ns & 1) ? ns >> 1 : -1;
                    if (eqm) {
                        pair_sums_df2<PSI, true>(SD, np, ptail, sa, lpa, tha, tla, qm, s_tab, acc_a);
                        if (nb) pair_sums_df2<PSI, true>(SD, np, ptail, sb, lpb, thb, tlb, qm, s_tab, acc_b);
                    } else {
                        pair_sums_df2<PSI, false>(SD, np, ptail, sa, lpa, tha, tla, qm, s_tab, acc_a);
                        if (nb) pair_sums_df2<PSI, false>(SD, np, ptail, sb, lpb, thb, tlb, qm, s_tab, acc_b);
                    }
                }
            }
            // the staged mass once per target less what it skipped: acc[4] = sum q
            if (sa == 0) acc_a[4] = mass - acc_a[4];
            else acc_a[4] = -acc_a[4];
            if (sb == 0) acc_b[4] = mass - acc_b[4];
            else acc_b[4] = -acc_b[4];
            // the sums of each target's lanes, in the order (x, y, z, q, log, ...) the finish takes
            dflt na_[NACC], nb_[NACC];
#pragma unroll
            for (int c = 0; c < NACC; ++c) {
                const int cc = c == 3 ? 4 : c == 4 ? 3 : c;     // 3 <- q (acc[4]), 4 <- log (acc[3])
                na_[c] = group_sum_dfl(dfl_norm(acc_a[cc]), lpa);
                nb_[c] = group_sum_dfl(dfl_norm(acc_b[cc]), lpb);
            }
            if (ADJ) {
                if (sa == 0) finish_target_adj_df<PSI>(A, G, L, ta, tha, tla, na_, s_tab, shift);
                if (act_b && sb == 0) finish_target_adj_df<PSI>(A, G, L, tbx, thb, tlb, nb_, s_tab, shift);
            } else {
                // the sums go to k_finish_df (one thread per target: the long double-float
                // L2P would leave the lanes of small target groups idle here)
                if (sa == 0) store_near_df(A, ta, leaf, na_);
                if (act_b && sb == 0) store_near_df(A, tbx, leaf, nb_);
            }
            tb += na + nb;
        }
    }
}

// Offsets for the mixed evaluation as FP32 (hi, lo) pairs, formed without FP64
// instructions (the difference to 2^-47): each sorted target from its leaf's
// centre, and each near leaf's centre from its target leaf's centre (one per
// direct-act pair).
__global__ void k_tgt_offsets(TreeView T, const int* __restrict__ leaves, int64_t n_cap, const int64_t* d_nl,
                              const double4_32a* __restrict__ tgt, float4* __restrict__ off)
{
    const int64_t n_leaves = dcount(d_nl, n_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp0; w < n_leaves; w += nw) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const int f = T.tfirst[node], n = T.tcount[node];
        for (int j = f + lane; j < f + n; j += 32) {
            const double4_32a x = tgt[j];
            const dflt dx = dfl_sub_exact(x.x, g[0]), dy = dfl_sub_exact(x.y, g[1]), dz = dfl_sub_exact(x.z, g[2]);
            off[2 * (size_t)j] = make_float4(dx.h, dy.h, dz.h, 0.f);
            off[2 * (size_t)j + 1] = make_float4(dx.l, dy.l, dz.l, 0.f);
        }
    }
}

// per direct-act pair: (hi offset, first source of the near leaf), (lo offset, its source count)
__global__ void k_pair_offsets(TreeView T, const uint64_t* __restrict__ tt, const uint32_t* __restrict__ ss,
                               int64_t n_cap, const int64_t* d_n, float4* __restrict__ dc)
{
    const int64_t n = dcount(d_n, n_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sl = ss[k];
        const double* gs = T.geom + (size_t)sl * GEOM_STRIDE;
        const double* gt = T.geom + (size_t)tt[k] * GEOM_STRIDE;
        const dflt dx = dfl_sub_exact(gs[0], gt[0]), dy = dfl_sub_exact(gs[1], gt[1]), dz = dfl_sub_exact(gs[2], gt[2]);
        dc[2 * k] = make_float4(dx.h, dy.h, dz.h, __int_as_float(T.first[sl]));
        dc[2 * k + 1] = make_float4(dx.l, dy.l, dz.l, __int_as_float(T.count[sl]));
    }
}

// Zero the leaf counter and size a persistent grid of 4-warp CTAs: up to
// per_sm per SM (the CTAs an SM holds at once); every warp takes target leaves
// from the counter until none are left, so uneven leaves leave no slot idle
// (CTAs beyond what the SMs hold start when others exit and find little or
// nothing left).
cudaError_t leaf_grid(unsigned long long* ctr, int64_t n_leaves, int per_sm, cudaStream_t s, int64_t* blocks)
{
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s)) || (e = cudaGetDevice(&dev)) ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    const int64_t want = (n_leaves + 3) / 4;
    *blocks = want < (int64_t)sms * per_sm ? want : (int64_t)sms * per_sm;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_eval32_prep(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                               const double4_32a* tgt, float4* toff, const uint64_t* p2p_t, const uint32_t* p2p_s,
                               int64_t n_p2p, const int64_t* d_np, float4* dc, cudaStream_t s)
{
    if (n_leaves > 0) {
        int64_t b = (n_leaves + 7) / 8;
        if (b > 152 * 64) b = 152 * 64;
        k_tgt_offsets<<<(unsigned)b, 256, 0, s>>>(T, leaves, n_leaves, d_nl, tgt, toff); count_launch();
    }
    if (n_p2p > 0) {
        int64_t b = (n_p2p + 255) / 256;
        if (b > 152 * 64) b = 152 * 64;
        k_pair_offsets<<<(unsigned)b, 256, 0, s>>>(T, p2p_t, p2p_s, n_p2p, d_np, dc); count_launch();
    }
    return cudaGetLastError();
}

// local/mpole: FP32 expansions, or double-float ones when dfar (the 1e-6 path)
cudaError_t launch_eval32(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* soff,
                          const float4* toff, const float4* dc, const double4_32a* tgt, const uint32_t* tperm, const int64_t* p2p_off,
                          const uint32_t* p2p_src, const void* local, const void* mpole, bool dfar, int p, int zero_mean,
                          double* psi, double* alpha, bool coincide, float4* nf, int* tleaf,
                          const void* frames, int64_t M, int what, unsigned long long* leaf_ctr, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    Eval32Args A;
    A.T = T;
    A.leaves = leaves;
    A.n_leaves = n_leaves;
    A.d_n_leaves = d_nl;
    A.soff = soff;
    A.toff = toff;
    A.dc = dc;
    A.tgt = tgt;
    A.tperm = tperm;
    A.p2p_off = p2p_off;
    A.p2p_src = p2p_src;
    A.local = dfar ? nullptr : static_cast<const float*>(local);
    A.base_mpole = dfar ? nullptr : static_cast<const float*>(mpole);
    A.local_df = dfar ? static_cast<const dflt*>(local) : nullptr;
    A.base_mpole_df = dfar ? static_cast<const dflt*>(mpole) : nullptr;
    A.p = p;
    A.want_psi = psi != nullptr;
    A.zero_mean = zero_mean;
    A.psi = psi;
    A.alpha = alpha;
    A.leaf_ctr = leaf_ctr;
    A.nf = nf;
    A.tleaf = tleaf;
    A.frames = static_cast<const FrameDF*>(frames);
    A.M = M;
    cudaError_t e;
    if (what & EVAL_NEAR) {
        int64_t blocks = 0;
        if ((e = leaf_grid(leaf_ctr, n_leaves, 7, s, &blocks))) return e;     // 7 per SM: __launch_bounds__
#define EVAL32_LAUNCH(PSI, MASK)                                                  \
        if (dfar) k_eval32<PSI, MASK, true><<<(unsigned)blocks, 128, 0, s>>>(A);  \
        else k_eval32<PSI, MASK, false><<<(unsigned)blocks, 128, 0, s>>>(A);
        if (coincide) {
            if (psi) { EVAL32_LAUNCH(true, true) }
            else { EVAL32_LAUNCH(false, true) }
        } else {
            if (psi) { EVAL32_LAUNCH(true, false) }
            else { EVAL32_LAUNCH(false, false) }
        }
#undef EVAL32_LAUNCH
        count_launch();
    }
    if (dfar && M > 0 && (what & EVAL_FINISH)) {
        int64_t fb = (M + 127) / 128;
        if (fb > 152 * 16) fb = 152 * 16;
        if (psi) k_finish_dfar<true><<<(unsigned)fb, 128, 0, s>>>(A);
        else k_finish_dfar<false><<<(unsigned)fb, 128, 0, s>>>(A);
        count_launch();
    }
    return cudaGetLastError();
}

// Table of the double-float logarithm: entry j < 128 holds log(c_j) and 1/c_j,
// c_j = 1 + j/128, each as an FP32 (hi, lo) pair rounded from FP64; entry 128
// holds log 2 as a 16-bit leading part and the FP32 rounding of the rest.
void fill_log_table(float* out)
{
    auto split = [](double v, float* hl) {
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
    };
    for (int j = 0; j < 128; ++j) {
        const double c = 1.0 + j / 128.0;
        split(std::log(c), out + 4 * j);
        split(1.0 / c, out + 4 * j + 2);
    }
    // log 2 with a 16-bit leading part: e times it is exact in FP32 for |e| < 2^7
    const double l2h = std::ldexp(std::nearbyint(std::ldexp(std::log(2.0), 16)), -16);
    out[4 * 128] = (float)l2h;
    out[4 * 128 + 1] = (float)(std::log(2.0) - l2h);
    out[4 * 128 + 2] = out[4 * 128 + 3] = 0.f;
}

cudaError_t launch_eval_df(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* soff,
                           const float4* toff, const float4* dc, const double4_32a* tgt, const uint32_t* tperm,
                           const int64_t* p2p_off, const uint32_t* p2p_src, const void* local, const void* mpole,
                           const float4* log_tab, int p, int zero_mean, double* psi, double* alpha,
                           const float4* doff, const void* w, int w_f32, double* grad3, float4* nf, int* tleaf,
                           const void* frames, int64_t M, int what, unsigned long long* leaf_ctr, cudaStream_t s)
{
    EvalDfArgs A;
    A.T = T;
    A.leaves = leaves;
    A.n_leaves = n_leaves;
    A.d_n_leaves = d_nl;
    A.soff = soff;
    A.toff = toff;
    A.dc = dc;
    A.tgt = tgt;
    A.tperm = tperm;
    A.p2p_off = p2p_off;
    A.p2p_src = p2p_src;
    A.local = static_cast<const dflt*>(local);
    A.base_mpole = static_cast<const dflt*>(mpole);
    A.log_tab = log_tab;
    A.p = p;
    A.zero_mean = zero_mean;
    A.psi = psi;
    A.alpha = alpha;
    A.leaf_ctr = leaf_ctr;
    A.doff = doff;
    A.w = w;
    A.w_f32 = w_f32;
    A.grad3 = grad3;
    A.nf = nf;
    A.tleaf = tleaf;
    A.frames = static_cast<const FrameDF*>(frames);
    A.M = M;
    cudaError_t e;
    if (n_leaves > 0 && (doff || (what & EVAL_NEAR))) {
        int64_t blocks = 0;
        if ((e = leaf_grid(leaf_ctr, n_leaves, 16, s, &blocks))) return e;
        if (doff) {                // the adjoint: near field and finish in one kernel
            if (psi) k_eval_df<true, true><<<(unsigned)blocks, 128, 0, s>>>(A);
            else k_eval_df<false, true><<<(unsigned)blocks, 128, 0, s>>>(A);
        } else {
            if (psi) k_eval_df<true, false><<<(unsigned)blocks, 128, 0, s>>>(A);
            else k_eval_df<false, false><<<(unsigned)blocks, 128, 0, s>>>(A);
        }
        count_launch();
    }
    if (!doff && M > 0 && (what & EVAL_FINISH)) {
        int64_t fb = (M + 127) / 128;
        if (fb > 152 * 16) fb = 152 * 16;
        if (psi) k_finish_df<true><<<(unsigned)fb, 128, 0, s>>>(A);
        else k_finish_df<false><<<(unsigned)fb, 128, 0, s>>>(A);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_count_pairs(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* p2p_off,
                               const uint32_t* p2p_src, unsigned long long* out, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    int64_t blocks = (n_leaves + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_count_pairs<<<(unsigned)blocks, 256, 0, s>>>(T, leaves, n_leaves, p2p_off, p2p_src, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const double4_32a* src,
                        const double4_32a* tgt,
                        const uint32_t* tperm, const int64_t* p2p_off, const uint32_t* p2p_src, const double* local,
                        const double* mpole, int p, int zero_mean, double sigma, double* psi, double* alpha,
                        double* gamma, double* mu, unsigned long long* leaf_ctr, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    EvalArgs A;
    A.T = T;
    A.leaves = leaves;
    A.n_leaves = n_leaves;
    A.d_n_leaves = d_nl;
    A.src = src;
    A.tgt = tgt;
    A.tperm = tperm;
    A.p2p_off = p2p_off;
    A.p2p_src = p2p_src;
    A.local = local;
    A.base_mpole = mpole;
    A.p = p;
    A.want_psi = psi != nullptr;
    A.zero_mean = zero_mean;
    A.psi = psi;
    A.alpha = alpha;
    A.gamma = gamma;
    A.mu = mu;
    A.npm_s = sin(0.5 * sigma) * sin(0.5 * sigma);
    A.leaf_ctr = leaf_ctr;
    int64_t blocks = 0;
    cudaError_t e;
    if ((e = leaf_grid(leaf_ctr, n_leaves, 16, s, &blocks))) return e;
    if (gamma) k_eval<true, false><<<(unsigned)blocks, 128, 0, s>>>(A);
    else if (sigma > 0.0) k_eval<false, true><<<(unsigned)blocks, 128, 0, s>>>(A);
    else k_eval<false, false><<<(unsigned)blocks, 128, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval_adj(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src,
                            const double4_32a* dip, const double4_32a* tgt, const uint32_t* tperm,
                            const int64_t* p2p_off, const uint32_t* p2p_src, const double* local, const double* mpole,
                            int p, int zero_mean, const void* w, int w_f32, double* phi, double* grad3,
                            unsigned long long* leaf_ctr, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    EvalAdjArgs AA;
    EvalArgs& A = AA.E;
    A.T = T;
    A.leaves = leaves;
    A.n_leaves = n_leaves;
    A.d_n_leaves = nullptr;
    A.src = src;
    A.tgt = tgt;
    A.tperm = tperm;
    A.p2p_off = p2p_off;
    A.p2p_src = p2p_src;
    A.local = local;
    A.base_mpole = mpole;
    A.p = p;
    A.want_psi = phi != nullptr;
    A.zero_mean = zero_mean;
    A.psi = phi;
    A.alpha = nullptr;
    A.gamma = nullptr;
    A.mu = nullptr;
    AA.dip = dip;
    AA.w = w;
    AA.w_f32 = w_f32;
    AA.grad3 = grad3;
    A.leaf_ctr = leaf_ctr;
    int64_t blocks = 0;
    cudaError_t e;
    if ((e = leaf_grid(leaf_ctr, n_leaves, 16, s, &blocks))) return e;
    k_eval_adj<<<(unsigned)blocks, 128, 0, s>>>(AA); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
