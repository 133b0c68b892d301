// Expansions: P2M (Lemma 1), M2M (Lemma 2), M2L (Lemma 3), L2L (Lemma 4), in
// FP64 (the FP64 path), FP32 (the mixed path) or double-float (pairs of FP32
// numbers on the FP32 pipe, the 1e-10 mixed path).
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
// The parameters (a, b, g, log k, ph1, ph2) depend only on the two box centres:
// they are formed once per M2L pair and once per parent-child link, in FP64
// (from centre differences), by k_pair_geo / k_child_geo; the translation
// kernels run in FP64 or FP32 from them.
#include "common.cuh"
#include "dfloat.cuh"
#include "xgeo.cuh"

namespace sfmm {

namespace {

constexpr double INV4PI = 0.079577471545947667884;   // 1/(4 pi)
constexpr double LOG2 = 0.69314718055994530942;

enum { K_M2M = 0, K_M2L = 1, K_L2L = 2 };

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

__device__ __forceinline__ XGeo make_geo(int kind, const double* gS, const double* gT)
{
    double sh, ch;
    cd eT, eS;
    pair_geometry(gS, gT, &sh, &ch, &eT, &eS);
    const double rS = gS[10], rT = gT[10];
    XGeo G;
    if (kind == K_M2L) {
        const double c = ch / sh;
        G.a = c * rS;
        G.b = c * rT;
        G.g = rS * rT / (sh * sh);          // (1 + c^2) r_S r_T
        G.logk = log(sh);
        G.p1x = eT.x; G.p1y = -eT.y;        // e^{-i phi_T}
        G.p2x = eS.x; G.p2y = -eS.y;        // e^{-i phi_S}
    } else if (kind == K_M2M) {
        const double t = sh / ch;
        G.a = t * rS;
        G.b = t / rT;
        G.g = (1.0 + t * t) * rS / rT;
        G.logk = log(ch);
        G.p1x = -eT.x; G.p1y = eT.y;        // -e^{-i phi_T}
        G.p2x = eS.x; G.p2y = eS.y;         //  e^{ i phi_S}
    } else {
        const double t = sh / ch;
        G.a = t / rS;
        G.b = t * rT;
        G.g = (1.0 + t * t) * rT / rS;
        G.logk = log(ch);
        G.p1x = eT.x; G.p1y = eT.y;         //  e^{ i phi_T}
        G.p2x = -eS.x; G.p2y = eS.y;        // -e^{-i phi_S}
    }
    return G;
}

__device__ __forceinline__ void store_geo(XGeo* out, const XGeo& G) { *out = G; }
__device__ __forceinline__ void store_geo(XGeoDF* out, const XGeo& G)
{
    XGeoDF D;
    D.a = dflt(G.a); D.b = dflt(G.b); D.g = dflt(G.g); D.logk = dflt(G.logk);
    D.p1x = dflt(G.p1x); D.p1y = dflt(G.p1y); D.p2x = dflt(G.p2x); D.p2y = dflt(G.p2y);
    *out = D;
}
// Mixed path: the same parameters computed in FP32 from the FP64 centre
// difference and sum (exact to rounding) and FP32 frame vectors; only the
// six centre differences/sums use the FP64 pipe.
__device__ __forceinline__ XGeo32 make_geo32(int kind, const double* gS, const double* gT, const float* fS,
                                             const float* fT)
{
    const float dx = (float)(gT[0] - gS[0]), dy = (float)(gT[1] - gS[1]), dz = (float)(gT[2] - gS[2]);
    const float sx = (float)(gT[0] + gS[0]), sy = (float)(gT[1] + gS[1]), sz = (float)(gT[2] + gS[2]);
    const float d2 = dx * dx + dy * dy + dz * dz, s2 = sx * sx + sy * sy + sz * sz;
    const float sh = 0.5f * sqrtf(d2), ch = 0.5f * sqrtf(s2);
    const bool anti = s2 < d2;
    const float vx = anti ? sx : dx, vy = anti ? sy : dy, vz = anti ? sz : dz;
    const float sg = anti ? 1.f : -1.f;
    float ux = vx * fS[0] + vy * fS[1] + vz * fS[2];
    float uy = vx * fS[3] + vy * fS[4] + vz * fS[5];
    float n2 = ux * ux + uy * uy;
    float eTx = 1.f, eTy = 0.f, eSx = 1.f, eSy = 0.f;
    if (n2 > 0.f) { const float inv = rsqrtf(n2); eTx = ux * inv; eTy = uy * inv; }
    ux = sg * (vx * fT[0] + vy * fT[1] + vz * fT[2]);
    uy = sg * (vx * fT[3] + vy * fT[4] + vz * fT[5]);
    n2 = ux * ux + uy * uy;
    if (n2 > 0.f) { const float inv = rsqrtf(n2); eSx = ux * inv; eSy = uy * inv; }
    const float rS = fS[6], rT = fT[6];
    XGeo32 H;
    if (kind == K_M2L) {
        const float c = ch / sh;
        H.a = c * rS; H.b = c * rT; H.g = rS * rT / (sh * sh); H.logk = logf(sh);
        H.p1x = eTx; H.p1y = -eTy; H.p2x = eSx; H.p2y = -eSy;
    } else if (kind == K_M2M) {
        const float t = sh / ch;
        H.a = t * rS; H.b = t / rT; H.g = (1.f + t * t) * rS / rT; H.logk = logf(ch);
        H.p1x = -eTx; H.p1y = eTy; H.p2x = eSx; H.p2y = eSy;
    } else {
        const float t = sh / ch;
        H.a = t / rS; H.b = t * rT; H.g = (1.f + t * t) * rT / rS; H.logk = logf(ch);
        H.p1x = eTx; H.p1y = eTy; H.p2x = -eSx; H.p2y = eSy;
    }
    H.ar = H.a * H.p1x; H.ai = H.a * H.p1y;
    H.br = H.b * H.p2x; H.bi = H.b * H.p2y;
    // rho = g/(a b) = 1/cos^2(theta/2) for M2L; its 32nd power must stay below 2^100
    const float ab = H.a * H.b;
    const bool big = !(ab > 0.f) || H.g > ab * 8.7f;
    H.rho = big ? 0.f : H.g / ab;
    H.big = big ? 1 : 0;
    H.pad[0] = H.pad[1] = 0.f;
    return H;
}

// FP32 frame vectors and scale of every node (e_theta, e_phi, r, padding)
__global__ void k_geom32(int n_nodes, const double* __restrict__ geom, float* __restrict__ g32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double* g = geom + (size_t)i * GEOM_STRIDE;
        float* o = g32 + (size_t)i * 8;
        for (int k = 0; k < 6; ++k) o[k] = (float)g[3 + k];
        o[6] = (float)g[10];
        o[7] = 0.f;
    }
}

__global__ void k_pair_geo32(TreeView T, const float* __restrict__ g32, const uint64_t* __restrict__ tt,
                             const uint32_t* __restrict__ ss, int64_t n_cap, const int64_t* d_n,
                             XGeo32* __restrict__ out)
{
    const int64_t n = dcount(d_n, n_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = ss[k], t = (uint32_t)tt[k];
        out[k] = make_geo32(K_M2L, T.geom + (size_t)s * GEOM_STRIDE, T.geom + (size_t)t * GEOM_STRIDE,
                            g32 + (size_t)s * 8, g32 + (size_t)t * 8);
    }
}

__global__ void k_child_geo32(TreeView T, const float* __restrict__ g32, XGeo32* __restrict__ m2m,
                              XGeo32* __restrict__ l2l)
{
    const int64_t nn = dcount(T.d_nn, T.n_nodes);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int par = T.parent[i];
        if (par < 0) continue;
        const double* gC = T.geom + (size_t)i * GEOM_STRIDE;
        const double* gP = T.geom + (size_t)par * GEOM_STRIDE;
        m2m[i] = make_geo32(K_M2M, gC, gP, g32 + (size_t)i * 8, g32 + (size_t)par * 8);
        l2l[i] = make_geo32(K_L2L, gP, gC, g32 + (size_t)par * 8, g32 + (size_t)i * 8);
    }
}

template <typename GR>
__global__ void k_pair_geo(TreeView T, const uint64_t* __restrict__ tt, const uint32_t* __restrict__ ss, int64_t n_cap,
                           const int64_t* d_n, GR* __restrict__ out)
{
    const int64_t n = dcount(d_n, n_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double* gS = T.geom + (size_t)ss[k] * GEOM_STRIDE;
        const double* gT = T.geom + (size_t)tt[k] * GEOM_STRIDE;
        store_geo(out + k, make_geo(K_M2L, gS, gT));
    }
}

// ------------------------------------------- double-float translation geometry
// The double-float paths form the translation parameters without FP64
// arithmetic (this GPU's FP64 pipe runs at 1/64 of the FP32 rate): the centre
// difference D = T - S and sum E = T + S are exact to 2^-47 from the FP64
// centres by integer arithmetic (dfl_sub_exact), the frames and scales are
// double-float copies made once per node (k_frame_df), and sqrt, quotients and
// log sin(theta/2) are double-float (the table logarithm of the evaluation).
// The azimuths come from the shorter of D and E as in pair_geometry.

__global__ void k_frame_df(int n_cap, const int64_t* d_nn, const double* __restrict__ geom, FrameDF* __restrict__ out)
{
    const int64_t n_nodes = dcount(d_nn, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double* g = geom + (size_t)i * GEOM_STRIDE;
        FrameDF F;
        for (int k = 0; k < 3; ++k) {
            F.et[k] = dflt(g[3 + k]);
            F.ep[k] = dflt(g[6 + k]);
        }
        F.r = dflt(g[10]);
        for (int k = 0; k < 3; ++k) F.c[k] = dflt(g[k]);
        out[i] = F;
    }
}

struct PairGeoDF {
    dflt sh, ch;             // sin, cos of half the angle between the centres
    dflt eTx, eTy, eSx, eSy; // e^{i phi_T^(S)}, e^{i phi_S^(T)}
};

__device__ __forceinline__ PairGeoDF pair_geometry_df(const double* gS, const double* gT, const FrameDF& FS,
                                                      const FrameDF& FT)
{
    const dflt dx = dfl_sub_exact(gT[0], gS[0]), dy = dfl_sub_exact(gT[1], gS[1]), dz = dfl_sub_exact(gT[2], gS[2]);
    const dflt ex = dfl_sub_exact(gT[0], -gS[0]), ey = dfl_sub_exact(gT[1], -gS[1]), ez = dfl_sub_exact(gT[2], -gS[2]);
    const dflt d2 = dx * dx + dy * dy + dz * dz;
    const dflt s2 = ex * ex + ey * ey + ez * ez;
    PairGeoDF P;
    P.sh = dfl_sqrt(d2) * 0.5f;
    P.ch = dfl_sqrt(s2) * 0.5f;
    const bool anti = s2.h < d2.h;
    const dflt vx = anti ? ex : dx, vy = anti ? ey : dy, vz = anti ? ez : dz;
    const float sg = anti ? 1.f : -1.f;
    const dflt one(1.f, 0.f), zero(0.f, 0.f);
    dflt ux = vx * FS.et[0] + vy * FS.et[1] + vz * FS.et[2];
    dflt uy = vx * FS.ep[0] + vy * FS.ep[1] + vz * FS.ep[2];
    dflt n = dfl_sqrt(ux * ux + uy * uy);
    if (n.h > 0.f) { P.eTx = ux / n; P.eTy = uy / n; } else { P.eTx = one; P.eTy = zero; }
    ux = (vx * FT.et[0] + vy * FT.et[1] + vz * FT.et[2]) * sg;
    uy = (vx * FT.ep[0] + vy * FT.ep[1] + vz * FT.ep[2]) * sg;
    n = dfl_sqrt(ux * ux + uy * uy);
    if (n.h > 0.f) { P.eSx = ux / n; P.eSy = uy / n; } else { P.eSx = one; P.eSy = zero; }
    return P;
}

// M2L parameters of the thread-per-pair double-float kernel (m2l_pair.cu):
// a ph1, b ph2, rho = g/(a b) = 1/cos^2(theta/2), log sin(theta/2).
__global__ void k_pair_geo_rho(TreeView T, const FrameDF* __restrict__ fr, const float4* __restrict__ log_tab,
                               const uint64_t* __restrict__ tt, const uint32_t* __restrict__ ss, int64_t n_cap,
                               const int64_t* d_n, XGeoRho* __restrict__ out)
{
    __shared__ float4 s_tab[129];
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = log_tab[i];
    __syncthreads();
    const int64_t n = dcount(d_n, n_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t si = ss[k], ti = (uint32_t)tt[k];
        const FrameDF FS = fr[si], FT = fr[ti];
        const PairGeoDF G = pair_geometry_df(T.geom + (size_t)si * GEOM_STRIDE, T.geom + (size_t)ti * GEOM_STRIDE,
                                             FS, FT);
        XGeoRho R;
        const dflt zero(0.f, 0.f);
        R.big = !(G.ch.h > 0.f) || G.ch.h * G.ch.h < 1.f / 8.7f;     // rho = 1/cos^2 > 8.7: near antipodes
        if (R.big) {
            R.ar = R.ai = R.br = R.bi = R.rho = R.logk = zero;
        } else {
            const dflt c = G.ch / G.sh;
            const dflt a = c * FS.r, b = c * FT.r;
            R.ar = a * G.eTx;                      // a e^{-i phi_T^(S)}
            R.ai = -(a * G.eTy);
            R.br = b * G.eSx;                      // b e^{-i phi_S^(T)}
            R.bi = -(b * G.eSy);
            R.rho = dflt(1.f, 0.f) / (G.ch * G.ch);
            R.logk = dfl_norm(dfl_log_lazy(G.sh, s_tab));
        }
        R.pad[0] = R.pad[1] = R.pad[2] = 0;
        out[k] = R;
    }
}

// M2M and L2L parameters per node with a parent (the double-float paths)
__global__ void k_child_geo_df(TreeView T, const FrameDF* __restrict__ fr, const float4* __restrict__ log_tab,
                               XGeoDF* __restrict__ m2m, XGeoDF* __restrict__ l2l)
{
    __shared__ float4 s_tab[129];
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = log_tab[i];
    __syncthreads();
    const int64_t nn = dcount(T.d_nn, T.n_nodes);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int par = T.parent[i];
        if (par < 0) continue;
        const double* gC = T.geom + (size_t)i * GEOM_STRIDE;
        const double* gP = T.geom + (size_t)par * GEOM_STRIDE;
        const FrameDF FC = fr[i], FP = fr[par];
        const dflt one(1.f, 0.f);
        {   // M2M: child (S) -> parent (T)
            const PairGeoDF G = pair_geometry_df(gC, gP, FC, FP);
            const dflt t = G.sh / G.ch;
            XGeoDF X;
            X.a = t * FC.r;
            X.b = t / FP.r;
            X.g = (one + t * t) * FC.r / FP.r;
            X.logk = dfl_log1m(G.sh * G.sh, s_tab) * 0.5f;     // log cos(theta/2)
            X.p1x = -G.eTx; X.p1y = G.eTy;         // -e^{-i phi_T}
            X.p2x = G.eSx; X.p2y = G.eSy;          //  e^{ i phi_S}
            m2m[i] = X;
        }
        {   // L2L: parent (S) -> child (T)
            const PairGeoDF G = pair_geometry_df(gP, gC, FP, FC);
            const dflt t = G.sh / G.ch;
            XGeoDF X;
            X.a = t / FP.r;
            X.b = t * FC.r;
            X.g = (one + t * t) * FC.r / FP.r;
            X.logk = dfl_log1m(G.sh * G.sh, s_tab) * 0.5f;     // log cos(theta/2)
            X.p1x = G.eTx; X.p1y = G.eTy;          //  e^{ i phi_T}
            X.p2x = -G.eSx; X.p2y = G.eSy;         // -e^{-i phi_S}
            l2l[i] = X;
        }
    }
}

// per node with a parent: child -> parent (M2M) and parent -> child (L2L)
template <typename GR>
__global__ void k_child_geo(TreeView T, GR* __restrict__ m2m, GR* __restrict__ l2l)
{
    const int64_t nn = dcount(T.d_nn, T.n_nodes);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int par = T.parent[i];
        if (par < 0) continue;
        const double* gC = T.geom + (size_t)i * GEOM_STRIDE;
        const double* gP = T.geom + (size_t)par * GEOM_STRIDE;
        store_geo(m2m + i, make_geo(K_M2M, gC, gP));
        store_geo(l2l + i, make_geo(K_L2L, gP, gC));
    }
}

// ------------------------------------------------------- warp translation
template <typename R> struct cx { R x, y; };
template <typename R> __device__ __forceinline__ cx<R> cmk(R x, R y) { cx<R> r; r.x = x; r.y = y; return r; }
template <typename R> __device__ __forceinline__ cx<R> cmul2(cx<R> a, cx<R> b)
{
    return cmk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float shfl_up(float v, int o) { return __shfl_up_sync(FULL, v, o); }
__device__ __forceinline__ double shfl_up(double v, int o) { return __shfl_up_sync(FULL, v, o); }
__device__ __forceinline__ dflt shfl_up(dflt v, int o) { return dfl_shfl_up(v, o); }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(FULL, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(FULL, v, o); }
__device__ __forceinline__ dflt shfl_xor(dflt v, int o) { return dfl_shfl_xor(v, o); }

// Inner products of the translations: acc += a b.  FP32/FP64 contract to one
// FMA; double-float accumulates lazily and is renormalised once after the loop.
__device__ __forceinline__ float mul_lazy(float a, float b) { return a * b; }
__device__ __forceinline__ double mul_lazy(double a, double b) { return a * b; }
__device__ __forceinline__ dflt mul_lazy(dflt a, dflt b) { return dfl_mul_lazy(a, b); }
__device__ __forceinline__ void mac(float& acc, float a, float b) { acc += a * b; }
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc += a * b; }
__device__ __forceinline__ void mac(dflt& acc, dflt a, dflt b) { dfl_mac(acc, a, b); }
__device__ __forceinline__ float renorm(float a) { return a; }
__device__ __forceinline__ double renorm(double a) { return a; }
__device__ __forceinline__ dflt renorm(dflt a) { return dfl_norm(a); }

// x^(lane+1) for every lane (inclusive prefix product)
template <typename R> __device__ __forceinline__ R warp_pow(R x, int lane)
{
    R v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const R t = shfl_up(v, o);
        if (lane >= o) v *= t;
    }
    return v;
}
template <typename R> __device__ __forceinline__ cx<R> warp_cpow(cx<R> x, int lane)
{
    cx<R> v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        cx<R> t;
        t.x = shfl_up(v.x, o);
        t.y = shfl_up(v.y, o);
        if (lane >= o) v = cmul2(v, t);
    }
    return v;
}
template <typename R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

template <typename R> struct WarpSmem {
    cx<R> u[PMAX];
    cx<R> w[PMAX];
    R apow[PMAX + 1];
    R bpow[PMAX + 1];
};

// Tables in shared memory, [k][lane]: T1[k][n-1] = C(n+k, n), T2[k][l-1] = C(l-1, k).
template <typename R> struct Tables {
    R t1[PMAX * PMAX];
    R t2[PMAX * PMAX];
};

template <typename R> __device__ __forceinline__ void load_tables(Tables<R>* st, const double* g)
{
    for (int i = threadIdx.x; i < 2 * PMAX * PMAX; i += blockDim.x) (&st->t1[0])[i] = (R)g[i];
    __syncthreads();
}

// One translation by the whole warp.  Input expansion (Cin, Qin, X = lane's
// coefficient); accumulates into (accC, accQ, accY).
template <typename R, typename GR>
__device__ __forceinline__ void warp_translate(int p, int lane, const GR& G, R Cin, R Qin, cx<R> X,
                                               const Tables<R>* tb, WarpSmem<R>* ws, R* accC, R* accQ, cx<R>* accY)
{
    const int l = lane + 1;
    const bool on = l <= p;
    const R ap = warp_pow<R>((R)G.a, lane), gp = warp_pow<R>((R)G.g, lane), bp = warp_pow<R>((R)G.b, lane);
    const cx<R> p1 = warp_cpow<R>(cmk<R>((R)G.p1x, (R)G.p1y), lane);
    const cx<R> p2 = warp_cpow<R>(cmk<R>((R)G.p2x, (R)G.p2y), lane);
    const cx<R> u = on ? cmul2(p1, X) : cmk<R>(0, 0);
    const R csum = warp_sum<R>(on ? ap * u.x : R(0));
    __syncwarp();
    ws->u[lane] = u;
    ws->apow[lane + 1] = ap;
    ws->bpow[lane + 1] = bp;
    if (lane == 0) { ws->apow[0] = R(1); ws->bpow[0] = R(1); }
    __syncwarp();
    cx<R> v = cmk<R>(0, 0);
    for (int k = 0; k <= p - l; ++k) {
        const R c = mul_lazy(tb->t1[k * PMAX + lane], ws->apow[k]);
        const cx<R> uu = ws->u[lane + k];
        mac(v.x, c, uu.x);
        mac(v.y, c, uu.y);
    }
    v = cmk<R>(renorm(v.x), renorm(v.y));
    ws->w[lane] = on ? cmk<R>(v.x * gp, v.y * gp) : cmk<R>(0, 0);
    __syncwarp();
    cx<R> o = cmk<R>(-Qin * bp / (R)l, R(0));
    for (int k = 0; k < l && on; ++k) {
        const R c = mul_lazy(tb->t2[k * PMAX + lane], ws->bpow[k]);
        const cx<R> ww = ws->w[lane - k];
        mac(o.x, c, ww.x);
        mac(o.y, c, ww.y);
    }
    o = cmk<R>(renorm(o.x), renorm(o.y));
    if (on) {
        const cx<R> y = cmul2(p2, o);
        accY->x += y.x;
        accY->y += y.y;
    }
    *accC += Cin + R(2) * Qin * (R)G.logk + R(2) * csum;
    *accQ += Qin;
    __syncwarp();
}

// ---------------------------------------------- pipelined list translation
// Lane l-1 of a translation spends p-l+1 terms on the first recurrence (v_l)
// and l terms on the second (Y_l), so each recurrence alone takes p lockstep
// steps although every lane has only p+1 terms in all.  For a list of
// translations into one expansion (the M2L list of a target box, the children
// of a parent in M2M) the second recurrence of translation i and the first of
// translation i+1 share one loop of p+1 steps: lane l takes its l terms of the
// second, then its p-l+1 terms of the first.  All lanes run one instruction
// stream; the operands are chosen per lane by index arithmetic:
//   binomial  tc[j][l-1] = C(l-1, j) for j < l, C(j, l) for j >= l (fixed),
//   power     pw[j] = b^j (second) or pw[33 + j - l] = a^(j-l) (first),
//   vector    vec[l-1-j] = w (second) or vec[32 + j - 1] = u (first).
template <typename R> struct FusedTables {
    R tc[(PMAX + 1) * PMAX];
};
template <typename R> struct FusedSmem {
    cx<R> vec[2 * PMAX];       // w of the pending translation, then u of the next
    R pw[2 * (PMAX + 1)];      // b^0..b^32 of the pending translation, then a^0..a^32 of the next
    cx<R> snap[PMAX];          // each lane's second-recurrence sum at its switch step
};

template <typename R> __device__ __forceinline__ void load_fused_tables(FusedTables<R>* st, const double* g)
{
    // g holds T1[k][n-1] = C(n+k, n) and T2[k][l-1] = C(l-1, k)
    for (int i = threadIdx.x; i < (PMAX + 1) * PMAX; i += blockDim.x) {
        const int j = i / PMAX, lane = i % PMAX, l = lane + 1;
        double v = 0.0;
        if (j < l) v = g[PMAX * PMAX + j * PMAX + lane];
        else if (j - l < PMAX) v = g[(j - l) * PMAX + lane];
        st->tc[i] = (R)v;
    }
    __syncthreads();
}

// Translations 0..n-1 of a list, accumulated into (accC, accQ, accY).
// fetch(i, &G, &C, &Q, &X) loads translation i's parameters and input.
template <typename R, typename GR, typename Fetch>
__device__ __forceinline__ void warp_translate_list(int p, int lane, int n, Fetch fetch, const FusedTables<R>* tb,
                                                    FusedSmem<R>* ws, R* accC, R* accQ, cx<R>* accY)
{
    const int l = lane + 1;
    const bool on = l <= p;
    cx<R> p2prev = cmk<R>(0, 0);                  // state of the translation whose second recurrence is pending
    R bpprev = 0, Qprev = 0;
    ws->vec[lane] = cmk<R>(0, 0);
    ws->pw[lane] = R(0);
    if (lane == 0) ws->pw[PMAX] = R(0);
    for (int i = 0; i <= n; ++i) {
        const bool has_next = i < n, has_prev = i > 0;
        R gp = 0, bp = 0, Q = 0;
        cx<R> p2 = cmk<R>(0, 0);
        if (has_next) {
            GR G;
            R C;
            cx<R> X;
            fetch(i, &G, &C, &Q, &X);
            const R ap = warp_pow<R>((R)G.a, lane);
            gp = warp_pow<R>((R)G.g, lane);
            bp = warp_pow<R>((R)G.b, lane);
            const cx<R> p1 = warp_cpow<R>(cmk<R>((R)G.p1x, (R)G.p1y), lane);
            p2 = warp_cpow<R>(cmk<R>((R)G.p2x, (R)G.p2y), lane);
            const cx<R> u = on ? cmul2(p1, X) : cmk<R>(0, 0);
            const R csum = warp_sum<R>(on ? ap * u.x : R(0));
            *accC += C + R(2) * Q * (R)G.logk + R(2) * csum;
            *accQ += Q;
            ws->vec[PMAX + lane] = u;
            ws->pw[PMAX + 2 + lane] = ap;
            if (lane == 0) ws->pw[PMAX + 1] = R(1);
        }
        __syncwarp();
        cx<R> acc = (has_prev && on) ? cmk<R>(-Qprev * bpprev / (R)l, R(0)) : cmk<R>(0, 0);
        const cx<R> zero = cmk<R>(0, 0);
        for (int j = 0; j <= p; ++j) {
            const bool second = j < l;
            if (j == l) { ws->snap[lane] = acc; acc = zero; }
            const R t = tb->tc[j * PMAX + lane];
            const R pw = ws->pw[second ? j : PMAX + 1 + j - l];
            const cx<R> vv = ws->vec[second ? lane - j : PMAX - 1 + j];
            const R c = mul_lazy(t, pw);
            mac(acc.x, c, vv.x);
            mac(acc.y, c, vv.y);
        }
        __syncwarp();
        if (has_prev && on) {
            const cx<R> o = ws->snap[lane];
            const cx<R> y = cmul2(p2prev, cmk<R>(renorm(o.x), renorm(o.y)));
            accY->x += y.x;
            accY->y += y.y;
        }
        if (has_next) {
            const cx<R> v = cmk<R>(renorm(acc.x), renorm(acc.y));
            ws->vec[lane] = on ? cmk<R>(v.x * gp, v.y * gp) : cmk<R>(0, 0);
            ws->pw[lane + 1] = bp;
            if (lane == 0) ws->pw[0] = R(1);
            p2prev = p2;
            bpprev = bp;
            Qprev = Q;
        }
        __syncwarp();
    }
}

template <typename R, typename ST>
__device__ __forceinline__ void load_exp(const ST* e, int lane, int p, R* C, R* Q, cx<R>* X)
{
    *C = (R)e[0];
    *Q = (R)e[1];
    *X = (lane < p) ? cmk<R>((R)e[2 + 2 * lane], (R)e[3 + 2 * lane]) : cmk<R>(0, 0);
}
// FP32 rows are 8-byte aligned (EXP_STRIDE floats = 264 bytes): one float2 load per coefficient
template <>
__device__ __forceinline__ void load_exp<float, float>(const float* e, int lane, int p, float* C, float* Q, cx<float>* X)
{
    const float2 cq = *reinterpret_cast<const float2*>(e);
    *C = cq.x;
    *Q = cq.y;
    if (lane < p) {
        const float2 x = *reinterpret_cast<const float2*>(e + 2 + 2 * lane);
        *X = cmk<float>(x.x, x.y);
    } else {
        *X = cmk<float>(0.f, 0.f);
    }
}

template <typename R, typename ST>
__device__ __forceinline__ void store_exp(ST* e, int lane, int p, R C, R Q, cx<R> Y, bool add)
{
    if (lane == 0) {
        if (add) { e[0] += (ST)C; e[1] += (ST)Q; } else { e[0] = (ST)C; e[1] = (ST)Q; }
    }
    if (lane < p) {
        if (add) { e[2 + 2 * lane] += (ST)Y.x; e[3 + 2 * lane] += (ST)Y.y; }
        else { e[2 + 2 * lane] = (ST)Y.x; e[3 + 2 * lane] = (ST)Y.y; }
    }
}

// atomic accumulation (leftover M2L pairs of the tensor-core kernel)
template <typename R, typename ST>
__device__ __forceinline__ void atomic_exp(ST* e, int lane, int p, R C, R Q, cx<R> Y)
{
    if (lane == 0) { atomicAdd(e, (ST)C); atomicAdd(e + 1, (ST)Q); }
    if (lane < p) { atomicAdd(e + 2 + 2 * lane, (ST)Y.x); atomicAdd(e + 3 + 2 * lane, (ST)Y.y); }
}

// ----------------------------------------------------------------- P2M
// FP64: from the key-sorted FP64 positions.
template <int P, typename ST>
__global__ void k_p2m(TreeView T, const int* __restrict__ leaves, int64_t n_cap, const int64_t* d_nl,
                      const double4_32a* __restrict__ src, ST* __restrict__ mpole)
{
    const int64_t n_leaves = dcount(d_nl, n_cap);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_leaves; w += (int64_t)gridDim.x * blockDim.x) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const double cx_ = g[0], cy = g[1], cz = g[2];
        const double inv_r = 1.0 / g[10];
        cd A[P];
#pragma unroll
        for (int l = 0; l < P; ++l) A[l] = mk(0.0, 0.0);
        double Csum = 0.0, Qsum = 0.0;
        const int f = T.first[node], n = T.count[node];
        for (int j = f; j < f + n; ++j) {
            const double4_32a y = src[j];
            const double dx = y.x - cx_, dy = y.y - cy, dz = y.z - cz;
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
        ST* e = mpole + (size_t)node * EXP_STRIDE;
        const double Q = INV4PI * Qsum;
        e[0] = ST(INV4PI * Csum - Q * LOG2);
        e[1] = ST(Q);
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const double s = -INV4PI / (double)(l + 1);
            e[2 + 2 * l] = ST(s * A[l].x);
            e[3 + 2 * l] = ST(s * A[l].y);
        }
        for (int l = P; l < PMAX; ++l) { e[2 + 2 * l] = ST(0.0); e[3 + 2 * l] = ST(0.0); }
    }
}

// Adjoint (FP64): charges h and tangent dipoles g at the sources.  A dipole's
// potential g . grad_x G(x, y) is the derivative of the point-mass potential
// along g, so its multipole is the derivative of Lemma 1 along g: with
// D = x - c, 1 + x.c = 2 - |D|^2/2 and z = (D.e_theta + i D.e_phi)/(1 + x.c),
//   dz = [(g.e_theta + i g.e_phi) - z (g.c)] / (1 + x.c),
//   dA_l = -(1/4pi) z^(l-1) dz,   dC = (1/4pi) (g.c)/(1 + x.c),   dQ = 0
// (d log cos^2(theta/2) = d log((1 + x.c)/2); x.g = 0).  Stored scaled like
// Lemma 1: A_l / r^l.
template <int P>
__global__ void k_p2m_adj(TreeView T, const int* __restrict__ leaves, int64_t n_leaves,
                          const double4_32a* __restrict__ src, const double4_32a* __restrict__ dip,
                          double* __restrict__ mpole)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_leaves; w += (int64_t)gridDim.x * blockDim.x) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const double cx_ = g[0], cy = g[1], cz = g[2];
        const double inv_r = 1.0 / g[10];
        cd A[P], B[P];
#pragma unroll
        for (int l = 0; l < P; ++l) { A[l] = mk(0.0, 0.0); B[l] = mk(0.0, 0.0); }
        double Csum = 0.0, Qsum = 0.0, Cdip = 0.0;
        const int f = T.first[node], n = T.count[node];
        for (int j = f; j < f + n; ++j) {
            const double4_32a y = src[j];
            const double4_32a gd = dip[j];
            const double dx = y.x - cx_, dy = y.y - cy, dz = y.z - cz;
            const double d2 = dx * dx + dy * dy + dz * dz;
            const double inv = 1.0 / (2.0 - 0.5 * d2);          // 1/(1 + x.c)
            const double zr = (dx * g[3] + dy * g[4] + dz * g[5]) * inv;
            const double zi = (dx * g[6] + dy * g[7] + dz * g[8]) * inv;
            const double gc = gd.x * cx_ + gd.y * cy + gd.z * cz;
            const double dzr = ((gd.x * g[3] + gd.y * g[4] + gd.z * g[5]) - zr * gc) * inv * inv_r;
            const double dzi = ((gd.x * g[6] + gd.y * g[7] + gd.z * g[8]) - zi * gc) * inv * inv_r;
            const cd zs = mk(zr * inv_r, zi * inv_r);
            const double h = y.w;
            Qsum += h;
            Csum += h * log1p(-0.25 * d2);
            Cdip += gc * inv;
            cd zp = mk(h, 0.0), zq = mk(dzr, dzi);
#pragma unroll
            for (int l = 0; l < P; ++l) {
                zp = cmul(zp, zs);
                A[l] = cadd(A[l], zp);          // h zs^(l+1)
                B[l] = cadd(B[l], zq);          // zs^l dzs
                zq = cmul(zq, zs);
            }
        }
        double* e = mpole + (size_t)node * EXP_STRIDE;
        const double Q = INV4PI * Qsum;
        e[0] = INV4PI * (Csum + Cdip) - Q * LOG2;
        e[1] = Q;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const double s = 1.0 / (double)(l + 1);
            e[2 + 2 * l] = -INV4PI * (s * A[l].x + B[l].x);
            e[3 + 2 * l] = -INV4PI * (s * A[l].y + B[l].y);
        }
        for (int l = P; l < PMAX; ++l) { e[2 + 2 * l] = 0.0; e[3 + 2 * l] = 0.0; }
    }
}

// Double-float (1e-10 mixed path): from each source's (hi, lo) offset to its
// leaf centre, z^l by repeated double-float products, log(1 - d^2/4) = 2 log
// cos(theta/2) by the table-driven double-float logarithm (tab: as in the
// evaluation).  One thread per leaf.
template <int P>
__global__ void __launch_bounds__(128) k_p2m_df(TreeView T, const int* __restrict__ leaves, int64_t n_leaves,
                                                const float4* __restrict__ off, const float4* __restrict__ log_tab,
                                                dflt* __restrict__ mpole)
{
    __shared__ float4 s_tab[129];
    for (int i = threadIdx.x; i < 129; i += blockDim.x) s_tab[i] = log_tab[i];
    __syncthreads();
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_leaves; w += (int64_t)gridDim.x * blockDim.x) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const dflt etx(g[3]), ety(g[4]), etz(g[5]), epx(g[6]), epy(g[7]), epz(g[8]);
        const dflt inv_r(1.0 / g[10]);
        dflt Ar[P], Ai[P];
#pragma unroll
        for (int l = 0; l < P; ++l) { Ar[l] = dflt(0.f, 0.f); Ai[l] = dflt(0.f, 0.f); }
        dflt Csum(0.f, 0.f), Qsum(0.f, 0.f);
        const int f = T.first[node], n = T.count[node];
        for (int j = f; j < f + n; ++j) {
            const float4 h = off[2 * (size_t)j], lo = off[2 * (size_t)j + 1];
            const dflt dx(h.x, lo.x), dy(h.y, lo.y), dz(h.z, lo.z), q(h.w, lo.w);
            const dflt d2 = dx * dx + dy * dy + dz * dz;
            const dflt sc = inv_r / (dflt(2.f, 0.f) - d2 * 0.5f);            // 1/(r (1 + y.c))
            const dflt zr = (dx * etx + dy * ety + dz * etz) * sc;
            const dflt zi = (dx * epx + dy * epy + dz * epz) * sc;
            Qsum += q;
            dfl_mac(Csum, q, dfl_log_lazy(dflt(1.f, 0.f) - d2 * 0.25f, s_tab));   // 2 log cos(theta/2)
            dflt pr = q, pi(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < P; ++l) {
                const dflt nr = pr * zr - pi * zi, ni = pr * zi + pi * zr;
                pr = nr;
                pi = ni;
                Ar[l] += pr;
                Ai[l] += pi;
            }
        }
        Csum = dfl_norm(Csum);
        dflt* e = mpole + (size_t)node * EXP_STRIDE;
        const dflt i4p(INV4PI), l2(LOG2);
        const dflt Q = i4p * Qsum;
        e[0] = i4p * Csum - Q * l2;
        e[1] = Q;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const dflt sl = -(i4p / dflt(l + 1));
            e[2 + 2 * l] = sl * Ar[l];
            e[3 + 2 * l] = sl * Ai[l];
        }
        for (int l = P; l < PMAX; ++l) { e[2 + 2 * l] = dflt(0.f, 0.f); e[3 + 2 * l] = dflt(0.f, 0.f); }
    }
}

// FP32: from each source's FP32 offset to its leaf centre (the recentring was
// done in FP64 when the offsets were formed).
template <int P>
__global__ void k_p2m32(TreeView T, const int* __restrict__ leaves, int64_t n_leaves, const float4* __restrict__ off,
                        float* __restrict__ mpole)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_leaves; w += (int64_t)gridDim.x * blockDim.x) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const float etx = (float)g[3], ety = (float)g[4], etz = (float)g[5];
        const float epx = (float)g[6], epy = (float)g[7], epz = (float)g[8];
        const float inv_r = (float)(1.0 / g[10]);
        cx<float> A[P];
#pragma unroll
        for (int l = 0; l < P; ++l) A[l] = cmk<float>(0.f, 0.f);
        float Csum = 0.f, Qsum = 0.f;
        const int f = T.first[node], n = T.count[node];
        for (int j = f; j < f + n; ++j) {
            const float4 y = off[2 * (size_t)j];
            const float d2 = y.x * y.x + y.y * y.y + y.z * y.z;
            const float sc = inv_r / (2.f - 0.5f * d2);
            const float zr = (y.x * etx + y.y * ety + y.z * etz) * sc;
            const float zi = (y.x * epx + y.y * epy + y.z * epz) * sc;
            Qsum += y.w;
            Csum += y.w * log1pf(-0.25f * d2);
            cx<float> zp = cmk<float>(y.w, 0.f);
#pragma unroll
            for (int l = 0; l < P; ++l) {
                zp = cmul2(zp, cmk<float>(zr, zi));
                A[l].x += zp.x;
                A[l].y += zp.y;
            }
        }
        float* e = mpole + (size_t)node * EXP_STRIDE;
        const float Q = (float)INV4PI * Qsum;
        e[0] = (float)INV4PI * Csum - Q * (float)LOG2;
        e[1] = Q;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const float s = -(float)INV4PI / (float)(l + 1);
            e[2 + 2 * l] = s * A[l].x;
            e[3 + 2 * l] = s * A[l].y;
        }
        for (int l = P; l < PMAX; ++l) { e[2 + 2 * l] = 0.f; e[3 + 2 * l] = 0.f; }
    }
}

// ----------------------------------------------------------------- M2M
// One warp per internal node of one level: sum of its children's multipoles
// (pipelined over the non-empty children).
template <typename R, typename GR, typename ST>
__global__ void k_m2m(TreeView T, int a, int b, int lvl, int p, const double* __restrict__ tables,
                      const GR* __restrict__ geo, ST* __restrict__ mpole)
{
    if (T.d_level) {              // graph mode: the parents are the nodes of level lvl
        a = (int)T.d_level[lvl];
        b = (int)T.d_level[lvl + 1];
    }
    __shared__ FusedTables<R> tb;
    __shared__ FusedSmem<R> ws[4];
    load_fused_tables<R>(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = a + (int64_t)blockIdx.x * 4 + wid; node < b; node += (int64_t)gridDim.x * 4) {
        const int c0 = T.child0[node];
        if (c0 < 0 || T.count[node] == 0) continue;
        unsigned mask = 0;                 // non-empty children
        for (int k = 0; k < 4; ++k)
            if (T.count[c0 + k] > 0) mask |= 1u << k;
        R accC = 0, accQ = 0;
        cx<R> accY = cmk<R>(0, 0);
        auto fetch = [&](int i, GR* G, R* C, R* Q, cx<R>* X) {
            const int c = c0 + (int)__fns(mask, 0, i + 1);
            *G = geo[c];
            load_exp<R>(mpole + (size_t)c * EXP_STRIDE, lane, p, C, Q, X);
        };
        warp_translate_list<R, GR>(p, lane, __popc(mask), fetch, &tb, &ws[wid], &accC, &accQ, &accY);
        store_exp<R>(mpole + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, false);
    }
}

// ----------------------------------------------------------------- M2L
// One warp per target box with a non-empty list; writes local = sum of M2Ls
// (pipelined over the list).
template <typename R, typename GR, typename ST>
__global__ void k_m2l(TreeView T, const int64_t* __restrict__ off, const uint32_t* __restrict__ srcs, int p,
                      const double* __restrict__ tables, const GR* __restrict__ geo, const ST* __restrict__ mpole,
                      ST* __restrict__ local)
{
    __shared__ FusedTables<R> tb;
    __shared__ FusedSmem<R> ws[4];
    load_fused_tables<R>(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = (int64_t)blockIdx.x * 4 + wid; node < T.n_nodes; node += (int64_t)gridDim.x * 4) {
        const int64_t lo = off[node], hi = off[node + 1];
        if (lo == hi) continue;
        R accC = 0, accQ = 0;
        cx<R> accY = cmk<R>(0, 0);
        auto fetch = [&](int i, GR* G, R* C, R* Q, cx<R>* X) {
            const int64_t k = lo + i;
            *G = geo[k];
            load_exp<R>(mpole + (size_t)srcs[k] * EXP_STRIDE, lane, p, C, Q, X);
        };
        warp_translate_list<R, GR>(p, lane, (int)(hi - lo), fetch, &tb, &ws[wid], &accC, &accQ, &accY);
        store_exp<R>(local + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, false);
    }
}

// ----------------------------------------------------------------- L2L
// One warp per node of one level holding targets: local += L2L(parent local).
template <typename R, typename GR, typename ST>
__global__ void k_l2l(TreeView T, int a, int b, int lvl, int p, const double* __restrict__ tables,
                      const GR* __restrict__ geo, ST* __restrict__ local)
{
    if (T.d_level) {              // graph mode: the nodes of level lvl
        a = (int)T.d_level[lvl];
        b = (int)T.d_level[lvl + 1];
    }
    __shared__ Tables<R> tb;
    __shared__ WarpSmem<R> ws[4];
    load_tables<R>(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t node = a + (int64_t)blockIdx.x * 4 + wid; node < b; node += (int64_t)gridDim.x * 4) {
        if (T.tcount[node] == 0) continue;
        const int par = T.parent[node];
        if (par < 0) continue;
        const GR G = geo[node];
        R C, Q;
        cx<R> X;
        load_exp<R>(local + (size_t)par * EXP_STRIDE, lane, p, &C, &Q, &X);
        R accC = 0, accQ = 0;
        cx<R> accY = cmk<R>(0, 0);
        warp_translate<R>(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        store_exp<R>(local + (size_t)node * EXP_STRIDE, lane, p, accC, accQ, accY, true);
    }
}

// ------------------------------------------------------ M2L, listed pairs
// One warp per pair of a list (the pairs the tensor-core M2L leaves out); the
// result is added atomically to the target's local expansion.
template <typename R, typename GR, typename ST>
__global__ void k_m2l_list(const uint64_t* __restrict__ ptgt, const uint32_t* __restrict__ psrc,
                           const uint32_t* __restrict__ list, const uint32_t* __restrict__ n_list, int p,
                           const double* __restrict__ tables, const GR* __restrict__ geo, const ST* __restrict__ mpole,
                           ST* __restrict__ local)
{
    __shared__ Tables<R> tb;
    __shared__ WarpSmem<R> ws[4];
    load_tables<R>(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = *n_list;
    for (int64_t w = (int64_t)blockIdx.x * 4 + wid; w < n; w += (int64_t)gridDim.x * 4) {
        const uint32_t k = list[w];
        const int s = (int)psrc[k], t = (int)ptgt[k];
        const GR G = geo[k];
        R C, Q;
        cx<R> X;
        load_exp<R>(mpole + (size_t)s * EXP_STRIDE, lane, p, &C, &Q, &X);
        R accC = 0, accQ = 0;
        cx<R> accY = cmk<R>(0, 0);
        warp_translate<R>(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        atomic_exp<R>(local + (size_t)t * EXP_STRIDE, lane, p, accC, accQ, accY);
    }
}

// M2L of the pairs the thread-per-pair double-float kernel leaves out (centres
// at or near antipodes): one warp per listed pair, in double-float from the
// a, b, g form, its parameters formed from the node centres in FP64; the
// result is added to the FP64 accumulators of the target box.
__global__ void k_m2l_left_df(TreeView T, const uint64_t* __restrict__ ptgt, const uint32_t* __restrict__ psrc,
                              const uint32_t* __restrict__ list, const uint32_t* __restrict__ n_list, int p,
                              const double* __restrict__ tables, const dflt* __restrict__ mpole,
                              double* __restrict__ acc)
{
    __shared__ Tables<dflt> tb;
    __shared__ WarpSmem<dflt> ws[4];
    load_tables<dflt>(&tb, tables);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = *n_list;
    for (int64_t w = (int64_t)blockIdx.x * 4 + wid; w < n; w += (int64_t)gridDim.x * 4) {
        const uint32_t k = list[w];
        const int s = (int)psrc[k], t = (int)ptgt[k];
        XGeoDF G;
        store_geo(&G, make_geo(K_M2L, T.geom + (size_t)s * GEOM_STRIDE, T.geom + (size_t)t * GEOM_STRIDE));
        dflt C, Q;
        cx<dflt> X;
        load_exp<dflt>(mpole + (size_t)s * EXP_STRIDE, lane, p, &C, &Q, &X);
        dflt accC(0.f, 0.f), accQ(0.f, 0.f);
        cx<dflt> accY = cmk<dflt>(dflt(0.f, 0.f), dflt(0.f, 0.f));
        warp_translate<dflt>(p, lane, G, C, Q, X, &tb, &ws[wid], &accC, &accQ, &accY);
        double* e = acc + (size_t)t * EXP_STRIDE;
        if (lane == 0) { atomicAdd(e, (double)accC); atomicAdd(e + 1, (double)accQ); }
        if (lane < p) { atomicAdd(e + 2 + 2 * lane, (double)accY.x); atomicAdd(e + 3 + 2 * lane, (double)accY.y); }
    }
}

// FP64 accumulators -> double-float expansions (every entry)
__global__ void k_acc_to_df(int64_t n, const double* __restrict__ acc, dflt* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dflt(acc[i]);
}

// FP32 offset of every key-sorted source from the centre of its leaf as an
// (hi, lo) pair (the difference to 2^-47, formed without FP64 instructions),
// plus its mass split the same way: off[2j] = (hi, q_hi), off[2j+1] = (lo, q_lo).
__global__ void k_src_offsets(TreeView T, const int* __restrict__ leaves, int64_t n_cap, const int64_t* d_nl,
                              const double4_32a* __restrict__ src, float4* __restrict__ off)
{
    const int64_t n_leaves = dcount(d_nl, n_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp0; w < n_leaves; w += nw) {
        const int node = leaves[w];
        const double* g = T.geom + (size_t)node * GEOM_STRIDE;
        const int f = T.first[node], n = T.count[node];
        for (int j = f + lane; j < f + n; j += 32) {
            const double4_32a y = src[j];
            const dflt dx = dfl_sub_exact(y.x, g[0]), dy = dfl_sub_exact(y.y, g[1]), dz = dfl_sub_exact(y.z, g[2]);
            const dflt q = dfl_sub_exact(y.w, 0.0);
            off[2 * (size_t)j] = make_float4(dx.h, dy.h, dz.h, q.h);
            off[2 * (size_t)j + 1] = make_float4(dx.l, dy.l, dz.l, q.l);
        }
    }
}

// Unscale for introspection: multipole A_l * r^l, local A_l / r^l.
template <typename ST>
__global__ void k_unscale(int n_nodes, const double* __restrict__ geom, const ST* __restrict__ in,
                          double* __restrict__ out, int p, int is_local)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = geom[(size_t)i * GEOM_STRIDE + 10];
        const ST* e = in + (size_t)i * EXP_STRIDE;
        double* o = out + (size_t)i * (2 * p + 2);
        o[0] = (double)e[0];
        o[1] = (double)e[1];
        double s = 1.0;
        for (int l = 0; l < p; ++l) {
            s = is_local ? s / r : s * r;
            o[2 + 2 * l] = (double)e[2 + 2 * l] * s;
            o[3 + 2 * l] = (double)e[3 + 2 * l] * s;
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

size_t xgeo_bytes(int ek) { return ek == EXP_F32 ? sizeof(XGeo32) : ek == EXP_DF ? sizeof(XGeoDF) : sizeof(XGeo); }

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

cudaError_t launch_geom32(int n_nodes, const double* geom, float* g32, cudaStream_t s)
{
    k_geom32<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, geom, g32); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pair_geo(const TreeView& T, const float* g32, const uint64_t* tt, const uint32_t* ss, int64_t n,
                            const int64_t* d_n, void* out, int ek, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (ek == EXP_F32) k_pair_geo32<<<grid_for(n, 256), 256, 0, s>>>(T, g32, tt, ss, n, d_n, static_cast<XGeo32*>(out));
    else if (ek == EXP_DF) k_pair_geo<XGeoDF><<<grid_for(n, 256), 256, 0, s>>>(T, tt, ss, n, d_n, static_cast<XGeoDF*>(out));
    else k_pair_geo<XGeo><<<grid_for(n, 256), 256, 0, s>>>(T, tt, ss, n, d_n, static_cast<XGeo*>(out));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_child_geo(const TreeView& T, const float* g32, void* m2m, void* l2l, int ek, cudaStream_t s)
{
    const unsigned g = grid_for(T.n_nodes, 256);
    if (ek == EXP_F32) k_child_geo32<<<g, 256, 0, s>>>(T, g32, static_cast<XGeo32*>(m2m), static_cast<XGeo32*>(l2l));
    else if (ek == EXP_DF) k_child_geo<XGeoDF><<<g, 256, 0, s>>>(T, static_cast<XGeoDF*>(m2m), static_cast<XGeoDF*>(l2l));
    else k_child_geo<XGeo><<<g, 256, 0, s>>>(T, static_cast<XGeo*>(m2m), static_cast<XGeo*>(l2l));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_src_offsets(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                               const double4_32a* src, float4* off, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    k_src_offsets<<<grid_for(n_leaves, 8), 256, 0, s>>>(T, leaves, n_leaves, d_nl, src, off); count_launch();
    return cudaGetLastError();
}

// mpole: double (FP64 path), float (mixed path) or double-float storage (1e-10 mixed path)
cudaError_t launch_p2m(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                       const double4_32a* src, const float4* off, const float4* log_tab, void* mpole, int p, int ek,
                       cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    const unsigned g = grid_for(n_leaves, 128);
#define P2M_CASE(PP)                                                                                       \
    case PP:                                                                                               \
        if (ek == EXP_F32) k_p2m32<PP><<<g, 128, 0, s>>>(T, leaves, n_leaves, off, static_cast<float*>(mpole)); \
        else if (ek == EXP_DF) k_p2m_df<PP><<<g, 128, 0, s>>>(T, leaves, n_leaves, off, log_tab, static_cast<dflt*>(mpole)); \
        else k_p2m<PP, double><<<g, 128, 0, s>>>(T, leaves, n_leaves, d_nl, src, static_cast<double*>(mpole)); \
        count_launch();                                                                                    \
        break;
    switch ((p + 3) / 4 * 4) {
        P2M_CASE(4) P2M_CASE(8) P2M_CASE(12) P2M_CASE(16) P2M_CASE(20) P2M_CASE(24) P2M_CASE(28) P2M_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef P2M_CASE
    return cudaGetLastError();
}

cudaError_t launch_p2m_adj(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src,
                           const double4_32a* dip, double* mpole, int p, cudaStream_t s)
{
    if (n_leaves == 0) return cudaSuccess;
    const unsigned g = grid_for(n_leaves, 128);
#define P2MA_CASE(PP)                                                                     \
    case PP:                                                                              \
        k_p2m_adj<PP><<<g, 128, 0, s>>>(T, leaves, n_leaves, src, dip, mpole);            \
        count_launch();                                                                   \
        break;
    switch ((p + 3) / 4 * 4) {
        P2MA_CASE(4) P2MA_CASE(8) P2MA_CASE(12) P2MA_CASE(16) P2MA_CASE(20) P2MA_CASE(24) P2MA_CASE(28) P2MA_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef P2MA_CASE
    return cudaGetLastError();
}

// parents a..b-1 (level lvl); graph mode: the bounds from the device, b - a the level-width capacity
cudaError_t launch_m2m(const TreeView& T, int a, int b, int lvl, int p, const double* tables, const void* geo,
                       void* mpole, int ek, cudaStream_t s)
{
    if (b <= a) return cudaSuccess;
    const unsigned g = grid_for(b - a, 4);
    if (ek == EXP_F32)
        k_m2m<float, XGeo32, float><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeo32*>(geo),
                                                      static_cast<float*>(mpole));
    else if (ek == EXP_DF)
        k_m2m<dflt, XGeoDF, dflt><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeoDF*>(geo),
                                                    static_cast<dflt*>(mpole));
    else
        k_m2m<double, XGeo, double><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeo*>(geo),
                                                      static_cast<double*>(mpole));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2l(const TreeView& T, const int64_t* off, const uint32_t* srcs, int p, const double* tables,
                       const void* geo, const void* mpole, void* local, int ek, cudaStream_t s)
{
    const unsigned g = grid_for(T.n_nodes, 4);
    if (ek == EXP_F32)
        k_m2l<float, XGeo32, float><<<g, 128, 0, s>>>(T, off, srcs, p, tables, static_cast<const XGeo32*>(geo),
                                                      static_cast<const float*>(mpole), static_cast<float*>(local));
    else if (ek == EXP_DF)
        k_m2l<dflt, XGeoDF, dflt><<<g, 128, 0, s>>>(T, off, srcs, p, tables, static_cast<const XGeoDF*>(geo),
                                                    static_cast<const dflt*>(mpole), static_cast<dflt*>(local));
    else
        k_m2l<double, XGeo, double><<<g, 128, 0, s>>>(T, off, srcs, p, tables, static_cast<const XGeo*>(geo),
                                                      static_cast<const double*>(mpole), static_cast<double*>(local));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2l_list(const uint64_t* ptgt, const uint32_t* psrc, const uint32_t* list, const uint32_t* n_list,
                            int64_t max_list, int p, const double* tables, const void* geo, const void* mpole,
                            void* local, cudaStream_t s)
{
    if (max_list == 0) return cudaSuccess;
    k_m2l_list<float, XGeo32, float><<<grid_for(max_list < 152 * 64 ? max_list : 152 * 64, 4), 128, 0, s>>>(
        ptgt, psrc, list, n_list, p, tables, static_cast<const XGeo32*>(geo), static_cast<const float*>(mpole),
        static_cast<float*>(local));
    count_launch();
    return cudaGetLastError();
}

size_t frame_df_bytes() { return sizeof(FrameDF); }

cudaError_t launch_frame_df(int n_nodes, const int64_t* d_nn, const double* geom, void* out, cudaStream_t s)
{
    if (n_nodes == 0) return cudaSuccess;
    k_frame_df<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, d_nn, geom, static_cast<FrameDF*>(out));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pair_geo_rho(const TreeView& T, const void* frames, const float4* log_tab, const uint64_t* tt,
                                const uint32_t* ss, int64_t n, const int64_t* d_n, void* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_pair_geo_rho<<<grid_for(n, 256), 256, 0, s>>>(T, static_cast<const FrameDF*>(frames), log_tab, tt, ss, n, d_n,
                                                     static_cast<XGeoRho*>(out));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_child_geo_df(const TreeView& T, const void* frames, const float4* log_tab, void* m2m, void* l2l,
                                cudaStream_t s)
{
    k_child_geo_df<<<grid_for(T.n_nodes, 256), 256, 0, s>>>(T, static_cast<const FrameDF*>(frames), log_tab,
                                                             static_cast<XGeoDF*>(m2m), static_cast<XGeoDF*>(l2l));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2l_left_df(const TreeView& T, const uint64_t* ptgt, const uint32_t* psrc, const uint32_t* list,
                               const uint32_t* n_list, int64_t max_list, int p, const double* tables,
                               const void* mpole, double* acc, cudaStream_t s)
{
    if (max_list == 0) return cudaSuccess;
    k_m2l_left_df<<<grid_for(max_list < 152 * 64 ? max_list : 152 * 64, 4), 128, 0, s>>>(
        T, ptgt, psrc, list, n_list, p, tables, static_cast<const dflt*>(mpole), acc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_acc_to_df(int64_t n, const double* acc, void* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_acc_to_df<<<grid_for(n, 256), 256, 0, s>>>(n, acc, static_cast<dflt*>(out));
    count_launch();
    return cudaGetLastError();
}

// nodes a..b-1 (level lvl); graph mode as launch_m2m
cudaError_t launch_l2l(const TreeView& T, int a, int b, int lvl, int p, const double* tables, const void* geo,
                       void* local, int ek, cudaStream_t s)
{
    if (b <= a) return cudaSuccess;
    const unsigned g = grid_for(b - a, 4);
    if (ek == EXP_F32)
        k_l2l<float, XGeo32, float><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeo32*>(geo),
                                                      static_cast<float*>(local));
    else if (ek == EXP_DF)
        k_l2l<dflt, XGeoDF, dflt><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeoDF*>(geo),
                                                    static_cast<dflt*>(local));
    else
        k_l2l<double, XGeo, double><<<g, 128, 0, s>>>(T, a, b, lvl, p, tables, static_cast<const XGeo*>(geo),
                                                      static_cast<double*>(local));
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_unscale(int n_nodes, const double* geom, const void* in, double* out, int p, int is_local,
                           int ek, cudaStream_t s)
{
    const unsigned g = grid_for(n_nodes, 256);
    if (ek == EXP_F32)
        k_unscale<float><<<g, 256, 0, s>>>(n_nodes, geom, static_cast<const float*>(in), out, p, is_local);
    else if (ek == EXP_DF)
        k_unscale<dflt><<<g, 256, 0, s>>>(n_nodes, geom, static_cast<const dflt*>(in), out, p, is_local);
    else
        k_unscale<double><<<g, 256, 0, s>>>(n_nodes, geom, static_cast<const double*>(in), out, p, is_local);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
