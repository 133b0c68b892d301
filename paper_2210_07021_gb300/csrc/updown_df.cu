// The up- and down-pass of the double-float far field (precision SFMM_MIXED
// and SFMM_MIXED_DF): P2M (Lemma 1) one warp per leaf and one lane per
// source, M2M (Lemma 2) and L2L (Lemma 4) one thread per translation.
//
// M2M and L2L use the general form of the translations (expand.cu):
//     u_l = ph1^l X_l,  v_n = sum_{l >= n} C(l, n) a^(l-n) u_l,  w_n = g^n v_n,
//     Y_l = ph2^l ( -Q b^l / l + sum_{n <= l} C(l-1, n-1) b^(l-n) w_n ),
//     C'  = C + 2 Q log k + 2 Re v_0,   Q' = Q,
// with both binomial sums as synthetic-division passes with multipliers a
// and b (dfops.cuh).  (The M2L kernel folds a and b into the vectors, which
// would underflow here: a = tan(theta/2) r_child is tiny at deep levels.)
// Each thread keeps its translation's vector in a row of shared memory between
// the O(p) diagonal steps (runtime loops) and the two unrolled passes, which
// run on (Re, Im) packed pairs (FP32x2 instructions).
//
// M2M: one thread per child of a level; the four children of a parent are
// consecutive (and aligned to four from the level's first node), so four
// neighbouring lanes hold the four translations into one parent and sum them
// from their rows.  L2L: one thread per node of a level holding targets; the
// node's local is its M2L sum (an FP64 accumulator) plus the parent's local
// translated.  Nodes of level 0 take their M2L sum alone.
#include "common.cuh"
#include "dfloat.cuh"
#include "dfops.cuh"
#include "xgeo.cuh"

namespace sfmm {

namespace {

constexpr int UW = 4;                 // warps per CTA
constexpr double INV4PI = 0.079577471545947667884;
constexpr double LOG2 = 0.69314718055994530942;

// One translation in the general form on the thread's row: in, X_l at
// row[2l], row[2l+1] (l = 1..p; the caller zeroes p < l <= P); out, Y_l there
// and C' in *Cout.
template <int P>
__device__ __forceinline__ void translate_row(dflt* row, int p, const XGeoDF& G, dflt C, dflt Q, dflt* Cout)
{
    {   // u_l = ph1^l X_l
        dflt zr = G.p1x, zi = G.p1y;
#pragma unroll 1
        for (int l = 1; l <= p; ++l) {
            if (l > 1) {
                dflt nr, ni;
                cmul_df(zr, zi, G.p1x, G.p1y, &nr, &ni);
                zr = nr;
                zi = ni;
            }
            cmul_df(zr, zi, row[2 * l], row[2 * l + 1], &row[2 * l], &row[2 * l + 1]);
        }
    }
    dflt v0;
    {   // both binomial stages on (Re, Im) packed pairs
        dflt2 c[P + 1];
        c[0] = dflt2{f2s(0.f), f2s(0.f)};
#pragma unroll
        for (int l = 1; l <= P; ++l) c[l] = ld_pair(row, l);
        pascal_up_mul2<P>(c, G.a);           // v = shifted by a
        v0 = renorm(dflt(c[0].h.x, c[0].l.x));
        dflt gp = G.g;                        // w_n = g^n v_n, at index n
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            c[n] = mul2_df(renorm2(c[n]), gp);
            if (n < P) gp = gp * G.g;
        }
        pascal_down_mul2<P>(c, G.b);         // o_l = sum C(l-1, n-1) b^(l-n) w_n
#pragma unroll
        for (int l = 1; l <= P; ++l) st_pair(row, l, renorm2(c[l]));
    }
    {   // Y_l = ph2^l (-Q b^l / l + o_l)
        dflt zr = G.p2x, zi = G.p2y, bp = G.b;
#pragma unroll 1
        for (int l = 1; l <= p; ++l) {
            if (l > 1) {
                dflt nr, ni;
                cmul_df(zr, zi, G.p2x, G.p2y, &nr, &ni);
                zr = nr;
                zi = ni;
                bp = bp * G.b;
            }
            const float fl = (float)l, il = 1.f / fl;
            const dflt qb = Q * bp;
            const float q1 = __fmul_rn(qb.h, il);                        // Q b^l / l
            const float rq = __fadd_rn(__fmaf_rn(-q1, fl, qb.h), qb.l);
            const dflt ql = dfl_fast_two_sum(q1, __fmul_rn(rq, il));
            const dflt orr = row[2 * l] - ql, oi = row[2 * l + 1];
            cmul_df(zr, zi, orr, oi, &row[2 * l], &row[2 * l + 1]);
        }
    }
    const dflt two(2.f, 0.f);
    *Cout = C + two * (Q * G.logk + v0);
}

__device__ __forceinline__ void ld_row(dflt* row, const dflt* e, int p, int P)
{
    for (int l = 1; l <= P; ++l) {
        if (l <= p) {
            const float4 v = *reinterpret_cast<const float4*>(e + 2 * l);
            row[2 * l] = dflt(v.x, v.y);
            row[2 * l + 1] = dflt(v.z, v.w);
        } else {
            row[2 * l] = dflt(0.f, 0.f);
            row[2 * l + 1] = dflt(0.f, 0.f);
        }
    }
}

// ----------------------------------------------------------------- M2M
template <int P>
__global__ void __launch_bounds__(128) k_m2m_df(TreeView T, int c0, int c1, int lvl, int p,
                                                const XGeoDF* __restrict__ geo, dflt* __restrict__ mpole)
{
    if (T.d_level) {              // graph mode: the children are the nodes of level lvl + 1
        c0 = (int)T.d_level[lvl + 1];
        c1 = (int)T.d_level[lvl + 2];
    }
    constexpr int RS = 2 * P + 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dflt* rows = reinterpret_cast<dflt*>(smem_raw);
    dflt* row = rows + threadIdx.x * RS;
    const int ncol = 2 * p + 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop bound is rounded up to whole sibling groups so that all four lanes of a group take part
    for (int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c - c0 < ((int64_t)(c1 - c0) + 31) / 32 * 32;
         c += stride) {
        const bool valid = c < c1;
        if (valid && T.count[c] > 0) {
            const dflt* e = mpole + (size_t)c * EXP_STRIDE;
            ld_row(row, e, p, P);
            dflt Cp;
            translate_row<P>(row, p, geo[c], e[0], e[1], &Cp);
            row[0] = Cp;
            row[1] = e[1];
        } else {
            for (int k = 0; k < ncol; ++k) row[k] = dflt(0.f, 0.f);
        }
        __syncwarp();
        // the four siblings' rows: lane r of the group sums columns r, r + 4, ... into the parent
        const int r = threadIdx.x & 3;
        const dflt* g0 = rows + (threadIdx.x & ~3) * RS;
        const int64_t first = c - r;              // the group's first child
        if (first < c1) {
            dflt* out = mpole + (size_t)T.parent[first] * EXP_STRIDE;
            for (int k = r; k < ncol; k += 4)
                out[k] = renorm(add_lazy(add_lazy(g0[k], g0[RS + k]), add_lazy(g0[2 * RS + k], g0[3 * RS + k])));
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- L2L
template <int P>
__global__ void __launch_bounds__(128) k_l2l_df(TreeView T, int a, int b, int lvl, int p,
                                                const XGeoDF* __restrict__ geo, const double* __restrict__ acc,
                                                dflt* __restrict__ local)
{
    if (T.d_level) {              // graph mode: the nodes of level lvl
        a = (int)T.d_level[lvl];
        b = (int)T.d_level[lvl + 1];
    }
    constexpr int RS = 2 * P + 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dflt* row = reinterpret_cast<dflt*>(smem_raw) + threadIdx.x * RS;
    const int ncol = 2 * p + 2;
    for (int64_t node = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < b;
         node += (int64_t)gridDim.x * blockDim.x) {
        const double* m = acc + (size_t)node * EXP_STRIDE;
        dflt* out = local + (size_t)node * EXP_STRIDE;
        if (T.tcount[node] == 0) {          // no target below: never evaluated; left at zero
            for (int k = 0; k < ncol; ++k) out[k] = dflt(0.f, 0.f);
            continue;
        }
        const int par = T.parent[node];
        if (par < 0) {
            for (int k = 0; k < ncol; ++k) out[k] = dflt(m[k]);
            continue;
        }
        const dflt* e = local + (size_t)par * EXP_STRIDE;
        ld_row(row, e, p, P);
        dflt Cp;
        translate_row<P>(row, p, geo[node], e[0], e[1], &Cp);
        row[0] = Cp;
        row[1] = e[1];
        for (int k = 0; k < ncol; ++k) out[k] = dflt(m[k]) + row[k];
    }
}

// ----------------------------------------------------------------- P2M
// One warp per leaf, one lane per source (in rounds of 32): z = tan(theta/2)
// e^{i phi} in the leaf frame from the source's (hi, lo) offset D,
// z = (D.e_theta + i D.e_phi) / (2 - |D|^2/2), scaled by 1/r; the lane's row
// holds q, q log(1 - |D|^2/4) = 2 q log cos(theta/2), and q z^l; lane k then
// sums columns k and k + 32 over the leaf's sources, and the multipole is
// Q = sum q / 4pi, C = (1/4pi) sum q log(..) - Q log 2, A_l = -(1/(4 pi l)) sum q z^l.
//
// DIP (the adjoint): each source also carries a tangent dipole g (doff: its
// (hi, lo) parts).  A dipole's potential is the derivative of the point mass's
// along g, so its multipole is Lemma 1 differentiated along g: with
// 1 + x.c = 2 - |D|^2/2, dz = [(g.e_theta + i g.e_phi) - z (g.c)] / (1 + x.c)
// (scaled by 1/r like z), dC = (1/4pi) (g.c) / (1 + x.c), dQ = 0 and
// dA_l = -(1/4pi) z^(l-1) dz; the row holds q z^l + l z^(l-1) dz for column l.
template <int P, bool DIP>
__global__ void __launch_bounds__(128) k_p2m_df_leaf(TreeView T, const int* __restrict__ leaves, int64_t n_cap,
                                                     const int64_t* d_nl, const float4* __restrict__ off,
                                                     const float4* __restrict__ doff,
                                                     const float4* __restrict__ log_tab, int p, dflt* __restrict__ mpole)
{
    const int64_t n_leaves = dcount(d_nl, n_cap);
    constexpr int RS = 2 * P + 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float4 s_tab[129];
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = log_tab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    dflt* rows = reinterpret_cast<dflt*>(smem_raw) + (size_t)wid * 32 * RS;
    dflt* row = rows + lane * RS;
    const int ncol = 2 * p + 2;
    for (int64_t w = (int64_t)blockIdx.x * UW + wid; w < n_leaves; w += (int64_t)gridDim.x * UW) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const dflt etx(g[3]), ety(g[4]), etz(g[5]), epx(g[6]), epy(g[7]), epz(g[8]);
        const dflt inv_r(1.0 / g[10]);
        const dflt ccx(g[0]), ccy(g[1]), ccz(g[2]);
        const int f = T.first[node], n = T.count[node];
        dflt sc[3] = {dflt(0.f, 0.f), dflt(0.f, 0.f), dflt(0.f, 0.f)};   // this lane's columns lane + 32 i (2p + 2 <= 66)
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            if (j < n) {
                const float4 h = off[2 * (size_t)(f + j)], lo = off[2 * (size_t)(f + j) + 1];
                const dflt dx(h.x, lo.x), dy(h.y, lo.y), dz(h.z, lo.z), q(h.w, lo.w);
                const dflt d2 = dx * dx + dy * dy + dz * dz;
                const dflt opc = dflt(2.f, 0.f) - d2 * 0.5f;                         // 1 + x.c
                const dflt inv = DIP ? dflt(1.f, 0.f) / opc : dflt(0.f, 0.f);
                const dflt sc = inv_r / opc;
                const dflt zr = (dx * etx + dy * ety + dz * etz) * sc;
                const dflt zi = (dx * epx + dy * epy + dz * epz) * sc;
                row[0] = q * dfl_norm(dfl_log_lazy(dflt(1.f, 0.f) - d2 * 0.25f, s_tab));
                row[1] = q;
                dflt pr = q, pi(0.f, 0.f);
                dflt qr(0.f, 0.f), qi(0.f, 0.f);     // z^(l-1) dz (DIP)
                if (DIP) {
                    const float4 gh = doff[2 * (size_t)(f + j)], gl = doff[2 * (size_t)(f + j) + 1];
                    const dflt gx(gh.x, gl.x), gy(gh.y, gl.y), gz(gh.z, gl.z);
                    const dflt gc = gx * ccx + gy * ccy + gz * ccz;
                    const dflt gci = gc * inv;
                    row[0] = row[0] + gci;
                    qr = (gx * etx + gy * ety + gz * etz) * sc - zr * gci;
                    qi = (gx * epx + gy * epy + gz * epz) * sc - zi * gci;
                }
#pragma unroll 1
                for (int l = 1; l <= p; ++l) {
                    dflt nr, ni;
                    cmul_df(pr, pi, zr, zi, &nr, &ni);
                    pr = nr;
                    pi = ni;
                    if (DIP) {
                        row[2 * l] = pr + qr * (float)l;
                        row[2 * l + 1] = pi + qi * (float)l;
                        cmul_df(qr, qi, zr, zi, &nr, &ni);
                        qr = nr;
                        qi = ni;
                    } else {
                        row[2 * l] = pr;
                        row[2 * l + 1] = pi;
                    }
                }
            }
            __syncwarp();
            const int nr = min(32, n - j0);
            // only the columns this lane owns (c < ncol < RS): every index stays below 32 RS
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (lane + 32 * i < ncol)
                    for (int r = 0; r < nr; ++r) sc[i] = add_lazy(sc[i], rows[r * RS + lane + 32 * i]);
            __syncwarp();
        }
        dflt* e = mpole + (size_t)node * EXP_STRIDE;
        const dflt i4p(INV4PI);
        // column k: 0 = sum q log(..), 1 = sum q, 2l / 2l+1 = sum q z^l (Re / Im)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int k = lane + 32 * i;
            if (k < ncol) {
                const dflt sk = renorm(sc[i]);
                e[k] = k < 2 ? i4p * sk : -(sk * (i4p / dflt(k >> 1)));
            }
        }
        __syncwarp();
        if (lane == 0) e[0] = e[0] - e[1] * dflt(LOG2);      // C = (1/4pi) sum q log(..) - Q log 2
        for (int k = ncol + lane; k < EXP_STRIDE; k += 32) e[k] = dflt(0.f, 0.f);
    }
}

inline unsigned grid_of(int64_t n, int per_block, int64_t cap)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

template <typename K>
cudaError_t smem_attr(K kern, size_t smem)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int P>
cudaError_t m2m_p(const TreeView& T, int c0, int c1, int lvl, int p, const void* geo, void* mpole, cudaStream_t s)
{
    const size_t smem = (size_t)128 * (2 * P + 3) * sizeof(dflt);
    cudaError_t e;
    if ((e = smem_attr(k_m2m_df<P>, smem))) return e;
    k_m2m_df<P><<<grid_of(c1 - c0, 128, 152 * 16), 128, smem, s>>>(T, c0, c1, lvl, p, static_cast<const XGeoDF*>(geo),
                                                                   static_cast<dflt*>(mpole));
    count_launch();
    return cudaGetLastError();
}

template <int P>
cudaError_t l2l_p(const TreeView& T, int a, int b, int lvl, int p, const void* geo, const double* acc, void* local,
                  cudaStream_t s)
{
    const size_t smem = (size_t)128 * (2 * P + 3) * sizeof(dflt);
    cudaError_t e;
    if ((e = smem_attr(k_l2l_df<P>, smem))) return e;
    k_l2l_df<P><<<grid_of(b - a, 128, 152 * 16), 128, smem, s>>>(T, a, b, lvl, p, static_cast<const XGeoDF*>(geo), acc,
                                                                 static_cast<dflt*>(local));
    count_launch();
    return cudaGetLastError();
}

template <int P>
cudaError_t p2m_p(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* off,
                  const float4* doff, const float4* log_tab, int p, void* mpole, cudaStream_t s)
{
    const size_t smem = (size_t)UW * 32 * (2 * P + 3) * sizeof(dflt);
    cudaError_t e;
    const unsigned grid = grid_of(n_leaves, UW, 152 * 32);
    if (doff) {
        if ((e = smem_attr(k_p2m_df_leaf<P, true>, smem))) return e;
        k_p2m_df_leaf<P, true><<<grid, UW * 32, smem, s>>>(T, leaves, n_leaves, d_nl, off, doff, log_tab, p,
                                                           static_cast<dflt*>(mpole));
    } else {
        if ((e = smem_attr(k_p2m_df_leaf<P, false>, smem))) return e;
        k_p2m_df_leaf<P, false><<<grid, UW * 32, smem, s>>>(T, leaves, n_leaves, d_nl, off, nullptr, log_tab, p,
                                                            static_cast<dflt*>(mpole));
    }
    count_launch();
    return cudaGetLastError();
}

#define SFMM_P_SWITCH(CALL)                                                                                 \
    switch ((p + 3) / 4 * 4) {                                                                              \
    case 4: return CALL(4); case 8: return CALL(8); case 12: return CALL(12); case 16: return CALL(16);     \
    case 20: return CALL(20); case 24: return CALL(24); case 28: return CALL(28); case 32: return CALL(32); \
    default: return cudaErrorInvalidValue;                                                                  \
    }

}  // namespace

// children c0..c1-1 (the nodes of level lvl + 1) -> their parents' multipoles.
// Graph mode (T.d_level set): the bounds are read on the device and c1 - c0 is
// the level-width capacity the launch is sized for.
cudaError_t launch_m2m_df(const TreeView& T, int c0, int c1, int lvl, int p, const void* geo, void* mpole,
                          cudaStream_t s)
{
    if (c1 <= c0) return cudaSuccess;
#define CALL(PP) m2m_p<PP>(T, c0, c1, lvl, p, geo, mpole, s)
    SFMM_P_SWITCH(CALL)
#undef CALL
}

// nodes a..b-1 (level lvl): local = M2L sum (acc) + L2L of the parent's local.
// Graph mode as for launch_m2m_df.
cudaError_t launch_l2l_df(const TreeView& T, int a, int b, int lvl, int p, const void* geo, const double* acc,
                          void* local, cudaStream_t s)
{
    if (b <= a) return cudaSuccess;
#define CALL(PP) l2l_p<PP>(T, a, b, lvl, p, geo, acc, local, s)
    SFMM_P_SWITCH(CALL)
#undef CALL
}

// doff: NULL, or the sources' tangent dipoles as (hi, lo) float4 pairs (the adjoint)
cudaError_t launch_p2m_df_leaf(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                               const float4* off, const float4* doff, const float4* log_tab, int p, void* mpole,
                               cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
#define CALL(PP) p2m_p<PP>(T, leaves, n_leaves, d_nl, off, doff, log_tab, p, mpole, s)
    SFMM_P_SWITCH(CALL)
#undef CALL
}

}  // namespace sfmm
