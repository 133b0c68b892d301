// Expansions: P2M (Lemma 1), M2M (Lemma 2), M2L (Lemma 3), L2L (Lemma 4), FP64.
//
// Storage.  An expansion is (C, Q, A_1..A_p) in the frame K_P of its box
// (zenith e_r(P), azimuth reference e_theta(P), Sec. 3.1), with the variable
// z = tan(theta/2) e^{i phi}.  For a point X and box centre c, writing
// D = X - c, the frame coordinates give z = (D.e_theta + i D.e_phi)/(1 + X.c)
// and 1 + X.c = 2 - |D|^2/2 (unit vectors): no trigonometry, and every
// quantity keeps its relative accuracy for close points.  Coefficients are
// stored scaled by the box scale r = tan(R/2): multipoles as A_l / r^l and
// locals as A_l r^l, so all stored values are O(1) at every level.
//
// Translations.  Lemmas 2-4 share one structure.  Writing
// T_{ll'}(x) = sum_n C(l-1,n-1) C(l',n) x^{l+l'-2n} (1+x^2)^n and folding the
// scales in, each becomes
//     u_l'  = ph1^l' X_l'                               (X: input coefficients)
//     v_n   = sum_{l' >= n} C(l', n) a^(l'-n) u_l'
//     w_n   = g^n v_n
//     Y_l   = ph2^l ( -Q b^l / l + sum_{n <= l} C(l-1, n-1) b^(l-n) w_n )
//     C'    = C + 2 Q log k + 2 Re sum_l a^l u_l,   Q' = Q
// with, for x = tan(theta/2) or cot(theta/2) of the centre-to-centre angle:
//     M2M  (Lemma 2): ph1 = -e^{-i phi_T^(S)}, ph2 = e^{ i phi_S^(T)}, a = t r_S,
//                     b = t / r_T, g = (1+t^2) r_S / r_T, k = cos(theta/2)
//     M2L  (Lemma 3): ph1 =  e^{-i phi_T^(S)}, ph2 = e^{-i phi_S^(T)}, a = c r_S,
//                     b = c r_T,  g = (1+c^2) r_S r_T,   k = sin(theta/2)
//     L2L  (Lemma 4): ph1 =  e^{ i phi_T^(S)}, ph2 = -e^{-i phi_S^(T)}, a = t / r_S,
//                     b = t r_T,  g = (1+t^2) r_T / r_S, k = cos(theta/2)
// which is the printed double sum evaluated in O(p^2) instead of O(p^3).
// One warp performs one translation; lane l-1 owns coefficient l (p <= 32).
#include "common.cuh"

namespace sfmm {

namespace {

constexpr double INV4PI = 0.079577471545947667884;   // 1/(4 pi)
constexpr double LOG2 = 0.69314718055994530942;

struct XGeo {
    double a, b, g, logk;
    cd ph1, ph2;
};

// Geometry of a translation from box S to box T (both rows of the geometry array).
// Returns sin(theta/2), cos(theta/2), e^{i phi_T^(S)}, e^{i phi_S^(T)}.
__device__ __forceinline__ void pair_geometry(const double* gS, const double* gT, double* sh, double* ch, cd* eT,
                                              cd* eS)
{
    const double dx = gT[0] - gS[0], dy = gT[1] - gS[1], dz = gT[2] - gS[2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    const double sx = gT[0] + gS[0], sy = gT[1] + gS[1], sz = gT[2] + gS[2];
    const double s2 = sx * sx + sy * sy + sz * sz;
    *sh = 0.5 * sqrt(d2);
    *ch = 0.5 * sqrt(s2);
    // The tangent part of T at S is the tangent part of D = T - S and also of
    // E = T + S; the tangent part of S at T is that of -D and of E.  Project
    // whichever of D, E is shorter (it is exact to rounding), so that both
    // azimuths come from one vector and stay consistent for nearly antipodal
    // centres, where only their sum matters (Lemma 3 at cot(theta/2) -> 0).
    const bool anti = s2 < d2;
    const double vx = anti ? sx : dx, vy = anti ? sy : dy, vz = anti ? sz : dz;
    const double sg = anti ? 1.0 : -1.0;
    // azimuth of T in K_S
    double ux = vx * gS[3] + vy * gS[4] + vz * gS[5];
    double uy = vx * gS[6] + vy * gS[7] + vz * gS[8];
    double n2 = ux * ux + uy * uy;
    // exactly antipodal centres (E = 0): e_theta(-S) = e_theta(S) and
    // e_phi(-S) = -e_phi(S), so the phase sum phi_T + phi_S is 0; take both as 1
    if (n2 > 0.0) { const double inv = rsqrt(n2); *eT = mk(ux * inv, uy * inv); }
    else *eT = mk(1.0, 0.0);
    // azimuth of S in K_T
    ux = sg * (vx * gT[3] + vy * gT[4] + vz * gT[5]);
    uy = sg * (vx * gT[6] + vy * gT[7] + vz * gT[8]);
    n2 = ux * ux + uy * uy;
    if (n2 > 0.0) { const double inv = rsqrt(n2); *eS = mk(ux * inv, uy * inv); }
    else *eS = mk(1.0, 0.0);
}

// x^(lane+1) for every lane (inclusive prefix product)
__device__ __forceinline__ double warp_pow(double x, int lane)
{
    double v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v *= t;
    }
    return v;
}
__device__ __forceinline__ cd warp_cpow(cd x, int lane)
{
    cd v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        cd t;
        t.x = __shfl_up_sync(FULL, v.x, o);
        t.y = __shfl_up_sync(FULL, v.y, o);
        if (lane >= o) v = cmul(v, t);
    }
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

struct WarpSmem {
    cd u[PMAX];
    cd w[PMAX];
    double apow[PMAX + 1];
    double bpow[PMAX + 1];
};

// Tables in shared memory, [k][lane]: T1[k][n-1] = C(n+k, n), T2[k][l-1] = C(l-1, k).
struct Tables {
    double t1[PMAX * PMAX];
    double t2[PMAX * PMAX];
};

__device__ __forceinline__ void load_tables(Tables* st, const double* g)
{
    for (int i = threadIdx.x; i < 2 * PMAX * PMAX; i += blockDim.x) (&st->t1[0])[i] = g[i];
    __syncthreads();
}

// One translation by the whole warp.  Input expansion (Cin, Qin, X = lane's
// coefficient); accumulates into (accC, accQ, accY).
__device__ __forceinline__ void warp_translate(int p, int lane, const XGeo& G, double Cin, double Qin, cd X,
                                               const Tables* tb, WarpSmem* ws, double* accC, double* accQ, cd* accY)
{
    const int l = lane + 1;
    const bool on = l <= p;
    const double ap = warp_pow(G.a, lane), gp = warp_pow(G.g, lane), bp = warp_pow(G.b, lane);
    const cd p1 = warp_cpow(G.ph1, lane), p2 = warp_cpow(G.ph2, lane);
    const cd u = on ? cmul(p1, X) : mk(0.0, 0.0);
    const double csum = warp_sum(on ? ap * u.x : 0.0);
    __syncwarp();
    ws->u[lane] = u;
    ws->apow[lane + 1] = ap;
    ws->bpow[lane + 1] = bp;
    if (lane == 0) { ws->apow[0] = 1.0; ws->bpow[0] = 1.0; }
    __syncwarp();
    cd v = mk(0.0, 0.0);
    for (int k = 0; k <= p - l; ++k) {
        const double c = tb->t1[k * PMAX + lane] * ws->apow[k];
        const cd uu = ws->u[lane + k];
        v.x += c * uu.x;
        v.y += c * uu.y;
    }
    ws->w[lane] = on ? cscale(v, gp) : mk(0.0, 0.0);
    __syncwarp();
    cd o = mk(-Qin * bp / (double)l, 0.0);
    for (int k = 0; k < l && on; ++k) {
        const double c = tb->t2[k * PMAX + lane] * ws->bpow[k];
        const cd ww = ws->w[lane - k];
        o.x += c * ww.x;
        o.y += c * ww.y;
    }
    if (on) *accY = cadd(*accY, cmul(p2, o));
    *accC += Cin + 2.0 * Qin * G.logk + 2.0 * csum;
    *accQ += Qin;
    __syncwarp();
}

__device__ __forceinline__ void load_exp(const double* e, int lane, int p, double* C, double* Q, cd* X)
{
    *C = e[0];
    *Q = e[1];
    *X = (lane < p) ? mk(e[2 + 2 * lane], e[3 + 2 * lane]) : mk(0.0, 0.0);
}

__device__ __forceinline__ void store_exp(double* e, int lane, int p, double C, double Q, cd Y, bool add)
{
    if (lane == 0) {
        if (add) { e[0] += C; e[1] += Q; } else { e[0] = C; e[1] = Q; }
    }
    if (lane < p) {
        if (add) { e[2 + 2 * lane] += Y.x; e[3 + 2 * lane] += Y.y; }
        else { e[2 + 2 * lane] = Y.x; e[3 + 2 * lane] = Y.y; }
    }
}

// ----------------------------------------------------------------- P2M
template <int P>
__global__ void k_p2m(TreeView T, const int* __restrict__ leaves, int64_t n_leaves, const double4_32a* __restrict__ src,
                      double* __restrict__ mpole)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_leaves; w += (int64_t)gridDim.x * blockDim.x) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const double cx = g[0], cy = g[1], cz = g[2];
        const double inv_r = 1.0 / g[10];
        cd A[P];
#pragma unroll
        for (int l = 0; l < P; ++l) A[l] = mk(0.0, 0.0);
        double Csum = 0.0, Qsum = 0.0;
        const int f = T.first[node], n = T.count[node];
        for (int j = f; j < f + n; ++j) {
            const double4_32a y = src[j];
            const double dx = y.x - cx, dy = y.y - cy, dz = y.z - cz;
            const double d2 = dx * dx + dy * dy + dz * dz;
            const double den = 2.0 - 0.5 * d2;   // 1 + y.c
            const double zr = (dx * g[3] + dy * g[4] + dz * g[5]) / den * inv_r;
            const double zi = (dx * g[6] + dy * g[7] + dz * g[8]) / den * inv_r;
            const double q = y.w;
            Qsum += q;
            Csum += q * log1p(-0.25 * d2);        // 2 log cos(theta/2)
            cd zp = mk(q, 0.0);
#pragma unroll
            for (int l = 0; l < P; ++l) {
                zp = cmul(zp, mk(zr, zi));
                A[l] = cadd(A[l], zp);
            }
        }
        double* e = mpole + (size_t)node * EXP_STRIDE;
        const double Q = INV4PI * Qsum;
        e[0] = INV4PI * Csum - Q * LOG2;
        e[1] = Q;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const double s = -INV4PI / (double)(l + 1);
            e[2 + 2 * l] = s * A[l].x;
            e[3 + 2 * l] = s * A[l].y;
        }
        for (int l = P; l < PMAX; ++l) { e[2 + 2 * l] = 0.0; e[3 + 2 * l] = 0.0; }
    }
}

// ----------------------------------------------------------------- M2M
// One warp per internal node of one level: sum of its 4 children's multipoles.
__global__ void k_m2m(TreeView T, int a, int b, int p, const double* __restrict__ tables, double* __restrict__ mpole)
{
    __shared__ Tables tb;
    __shared__ WarpSmem ws[4];
    load_tables(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = a + (int64_t)blockIdx.x * 4 + wid; node < b; node += (int64_t)gridDim.x * 4) {
        const int c0 = T.child0[node];
        if (c0 < 0 || T.count[node] == 0) continue;
        double accC = 0.0, accQ = 0.0;
        cd accY = mk(0.0, 0.0);
        const double* gT = T.geom + (size_t)node * GEOM_STRIDE;
        for (int c = c0; c < c0 + 4; ++c) {
            if (T.count[c] == 0) continue;
            const double* gS = T.geom + (size_t)c * GEOM_STRIDE;
            double sh, ch;
            cd eT, eS;
            pair_geometry(gS, gT, &sh, &ch, &eT, &eS);
            const double t = sh / ch;
            XGeo G;
            G.a = t * gS[10];
            G.b = t / gT[10];
            G.g = (1.0 + t * t) * gS[10] / gT[10];
            G.logk = log(ch);
            G.ph1 = mk(-eT.x, eT.y);          // -e^{-i phi_T}
            G.ph2 = eS;                       //  e^{ i phi_S}
            double C, Q;
            cd X;
            load_exp(mpole + (size_t)c * EXP_STRIDE, lane, p, &C, &Q, &X);
            warp_translate(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        }
        store_exp(mpole + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, false);
        if (lane < PMAX - p) { }  // coefficients above p stay as written by P2M / zero-init
    }
}

// ----------------------------------------------------------------- M2L
// One warp per target box with a non-empty list; writes local = sum of M2Ls.
__global__ void k_m2l(TreeView T, const int64_t* __restrict__ off, const uint32_t* __restrict__ srcs, int p,
                      const double* __restrict__ tables, const double* __restrict__ mpole, double* __restrict__ local)
{
    __shared__ Tables tb;
    __shared__ WarpSmem ws[4];
    load_tables(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = (int64_t)blockIdx.x * 4 + wid; node < T.n_nodes; node += (int64_t)gridDim.x * 4) {
        const int64_t lo = off[node], hi = off[node + 1];
        if (lo == hi) continue;
        double accC = 0.0, accQ = 0.0;
        cd accY = mk(0.0, 0.0);
        const double* gT = T.geom + (size_t)node * GEOM_STRIDE;
        for (int64_t k = lo; k < hi; ++k) {
            const int s = (int)srcs[k];
            const double* gS = T.geom + (size_t)s * GEOM_STRIDE;
            double sh, ch;
            cd eT, eS;
            pair_geometry(gS, gT, &sh, &ch, &eT, &eS);
            const double c = ch / sh;
            XGeo G;
            G.a = c * gS[10];
            G.b = c * gT[10];
            G.g = gS[10] * gT[10] / (sh * sh);  // (1 + c^2) r_S r_T
            G.logk = log(sh);
            G.ph1 = cconj(eT);                   // e^{-i phi_T}
            G.ph2 = cconj(eS);                   // e^{-i phi_S}
            double C, Q;
            cd X;
            load_exp(mpole + (size_t)s * EXP_STRIDE, lane, p, &C, &Q, &X);
            warp_translate(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        }
        store_exp(local + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, false);
    }
}

// ----------------------------------------------------------------- L2L
// One warp per node of one level holding targets: local += L2L(parent local).
__global__ void k_l2l(TreeView T, int a, int b, int p, const double* __restrict__ tables, double* __restrict__ local)
{
    __shared__ Tables tb;
    __shared__ WarpSmem ws[4];
    load_tables(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = a + (int64_t)blockIdx.x * 4 + wid; node < b; node += (int64_t)gridDim.x * 4) {
        if (T.tcount[node] == 0) continue;
        const int par = T.parent[node];
        if (par < 0) continue;
        const double* gS = T.geom + (size_t)par * GEOM_STRIDE;
        const double* gT = T.geom + (size_t)node * GEOM_STRIDE;
        double sh, ch;
        cd eT, eS;
        pair_geometry(gS, gT, &sh, &ch, &eT, &eS);
        const double t = sh / ch;
        XGeo G;
        G.a = t / gS[10];
        G.b = t * gT[10];
        G.g = (1.0 + t * t) * gT[10] / gS[10];
        G.logk = log(ch);
        G.ph1 = eT;                          //  e^{ i phi_T}
        G.ph2 = mk(-eS.x, eS.y);             // -e^{-i phi_S}
        double C, Q;
        cd X;
        load_exp(local + (size_t)par * EXP_STRIDE, lane, p, &C, &Q, &X);
        double accC = 0.0, accQ = 0.0;
        cd accY = mk(0.0, 0.0);
        warp_translate(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        store_exp(local + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, true);
    }
}

// Unscale for introspection: multipole A_l * r^l, local A_l / r^l.
__global__ void k_unscale(int n_nodes, const double* __restrict__ geom, const double* __restrict__ in,
                          double* __restrict__ out, int p, int is_local)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = geom[(size_t)i * GEOM_STRIDE + 10];
        const double* e = in + (size_t)i * EXP_STRIDE;
        double* o = out + (size_t)i * (2 * p + 2);
        o[0] = e[0];
        o[1] = e[1];
        double s = 1.0;
        for (int l = 0; l < p; ++l) {
            s = is_local ? s / r : s * r;
            o[2 + 2 * l] = e[2 + 2 * l] * s;
            o[3 + 2 * l] = e[3 + 2 * l] * s;
        }
    }
}

inline unsigned grid_for(int64_t n, int per_block)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)b;
}

}  // namespace

void fill_tables(double* h)   // [2][PMAX][PMAX]
{
    double C[2 * PMAX + 2][2 * PMAX + 2] = {};
    for (int n = 0; n < 2 * PMAX + 2; ++n) {
        C[n][0] = 1.0;
        for (int k = 1; k <= n; ++k) C[n][k] = C[n - 1][k - 1] + (k <= n - 1 ? C[n - 1][k] : 0.0);
    }
    for (int k = 0; k < PMAX; ++k)
        for (int lane = 0; lane < PMAX; ++lane) {
            const int n = lane + 1;
            h[k * PMAX + lane] = C[n + k][n];
            h[PMAX * PMAX + k * PMAX + lane] = (k <= lane) ? C[lane][k] : 0.0;
        }
}

cudaError_t launch_p2m(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src, double* mpole, int p,
                       cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    const unsigned g = grid_for(n_leaves, 128);
#define P2M_CASE(PP) case PP: k_p2m<PP><<<g, 128, 0, s>>>(T, leaves, n_leaves, src, mpole); count_launch(); break;
    switch ((p + 3) / 4 * 4) {
        P2M_CASE(4) P2M_CASE(8) P2M_CASE(12) P2M_CASE(16) P2M_CASE(20) P2M_CASE(24) P2M_CASE(28) P2M_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef P2M_CASE
    return cudaGetLastError();
}

cudaError_t launch_m2m(const TreeView& T, int a, int b, int p, const double* tables, double* mpole, cudaStream_t s)
{
    if (b <= a) return cudaSuccess;
    k_m2m<<<grid_for(b - a, 4), 128, 0, s>>>(T, a, b, p, tables, mpole); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2l(const TreeView& T, const int64_t* off, const uint32_t* srcs, int p, const double* tables,
                       const double* mpole, double* local, cudaStream_t s)
{
    k_m2l<<<grid_for(T.n_nodes, 4), 128, 0, s>>>(T, off, srcs, p, tables, mpole, local); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_l2l(const TreeView& T, int a, int b, int p, const double* tables, double* local, cudaStream_t s)
{
    if (b <= a) return cudaSuccess;
    k_l2l<<<grid_for(b - a, 4), 128, 0, s>>>(T, a, b, p, tables, local); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_unscale(int n_nodes, const double* geom, const double* in, double* out, int p, int is_local,
                           cudaStream_t s)
{
    k_unscale<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, geom, in, out, p, is_local); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
