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
// One warp per target leaf.  The leaf's targets are taken in groups of tpw
// (a power of two >= the target count, at most 32); each target gets
// 32/tpw lanes that split its sources and are combined by xor shuffles.
#include "common.cuh"

namespace sfmm {

namespace {

constexpr double INV4PI = 0.079577471545947667884;
constexpr double INV2PI = 0.15915494309189533577;
constexpr double LOG2 = 0.69314718055994530942;
constexpr double LOG4 = 1.3862943611198906188;

struct EvalArgs {
    TreeView T;
    const int* leaves;        // target leaves (tcount > 0)
    int64_t n_leaves;
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
};

__device__ __forceinline__ double group_sum(double v, int lpt)
{
    for (int o = lpt >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__global__ void __launch_bounds__(128) k_eval(EvalArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double shift = 0.0;
    if (A.zero_mean)
        for (int b = 0; b < 12; ++b) shift += A.base_mpole[(size_t)b * EXP_STRIDE + 1];
    for (int64_t w = warp0; w < A.n_leaves; w += nwarps) {
        const int leaf = A.leaves[w];
        const int tf = A.T.tfirst[leaf], tc = A.T.tcount[leaf];
        const double* g = A.T.geom + (size_t)leaf * GEOM_STRIDE;
        const double* L = A.local + (size_t)leaf * EXP_STRIDE;
        const int64_t nb0 = A.p2p_off[leaf], nb1 = A.p2p_off[leaf + 1];
        int tpw = 1;
        while (tpw < tc && tpw < 32) tpw <<= 1;
        const int lpt = 32 / tpw;
        const int slot = lane / lpt, sub = lane % lpt;
        for (int tb = 0; tb < tc; tb += tpw) {
            const int ti = tb + slot;
            const bool active = ti < tc;
            const double4_32a x = A.tgt[tf + (active ? ti : 0)];
            double sl = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, sq = 0.0;
            for (int64_t k = nb0; k < nb1; ++k) {
                const int sleaf = (int)A.p2p_src[k];
                const int f = A.T.first[sleaf], n = A.T.count[sleaf];
                for (int j = f + sub; j < f + n; j += lpt) {
                    const double4_32a y = A.src[j];
                    const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 > 0.0) {
                        const double wq = y.w / d2;
                        sx += wq * dx;
                        sy += wq * dy;
                        sz += wq * dz;
                        sq += y.w;
                        if (A.want_psi) sl += y.w * log(d2);
                    }
                }
            }
            sx = group_sum(sx, lpt);
            sy = group_sum(sy, lpt);
            sz = group_sum(sz, lpt);
            sq = group_sum(sq, lpt);
            if (A.want_psi) sl = group_sum(sl, lpt);
            if (!active || sub != 0) continue;
            // ---- L2P in the leaf frame
            const double Dx = x.x - g[0], Dy = x.y - g[1], Dz = x.z - g[2];
            const double D2 = Dx * Dx + Dy * Dy + Dz * Dz;
            const double den = 2.0 - 0.5 * D2;                  // 1 + x.c
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
            a3x += INV2PI * (sx - 0.5 * x.x * sq);
            a3y += INV2PI * (sy - 0.5 * x.y * sq);
            a3z += INV2PI * (sz - 0.5 * x.z * sq);
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

}  // namespace

cudaError_t launch_count_pairs(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* p2p_off,
                               const uint32_t* p2p_src, unsigned long long* out, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    int64_t blocks = (n_leaves + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_count_pairs<<<(unsigned)blocks, 256, 0, s>>>(T, leaves, n_leaves, p2p_off, p2p_src, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src, const double4_32a* tgt,
                        const uint32_t* tperm, const int64_t* p2p_off, const uint32_t* p2p_src, const double* local,
                        const double* mpole, int p, int zero_mean, double* psi, double* alpha, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    EvalArgs A;
    A.T = T;
    A.leaves = leaves;
    A.n_leaves = n_leaves;
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
    int64_t blocks = (n_leaves + 3) / 4;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_eval<<<(unsigned)blocks, 128, 0, s>>>(A); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
