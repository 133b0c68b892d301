// Translation parameters (Lemmas 2-4) shared by the translation kernels.
//
// For a translation from box S to box T, with x = tan(theta/2) (M2M, L2L) or
// cot(theta/2) (M2L) of the centre-to-centre angle and the scales r = tan(R/2)
// of the two boxes, the translated scaled coefficients are
//     u_l' = ph1^l' X_l',  v_n = sum_{l' >= n} C(l', n) a^(l'-n) u_l',  w_n = g^n v_n,
//     Y_l  = ph2^l ( -Q b^l / l + sum_{n <= l} C(l-1, n-1) b^(l-n) w_n ),
//     C'   = C + 2 Q log k + 2 Re sum_l a^l u_l,   Q' = Q
// (expand.cu derives a, b, g, k, ph1, ph2 per lemma).
#pragma once
#include "dfloat.cuh"

namespace sfmm {

// A node's frame in double-float, rounded from FP64 once per node (k_frame_df):
// e_theta, e_phi, the scale r = tan(R/2) and the centre c.
struct __align__(16) FrameDF {
    dflt et[3], ep[3], r, c[3];
};

// 64 bytes of translation parameters, formed in FP64.
struct __align__(16) XGeo {
    double a, b, g, logk;
    double p1x, p1y, p2x, p2y;
};

// The same parameters rounded to FP32 for the FP32 path, plus the fields of
// the tensor-core M2L (u = (a ph1)^l X, Y = (b ph2)^l ..., rho = g/(a b)):
// big = 1 when rho^32 exceeds 2^100 (centres near antipodes).
struct __align__(16) XGeo32 {
    float a, b, g, logk;
    float p1x, p1y, p2x, p2y;
    float ar, ai, br, bi;
    float rho;
    int big;
    float pad[2];
};

// The FP64 parameters rounded to double-float pairs.
struct __align__(16) XGeoDF {
    dflt a, b, g, logk;
    dflt p1x, p1y, p2x, p2y;
};

// M2L parameters of the thread-per-pair double-float kernel (m2l_pair.cu), formed
// in FP64 and rounded to double-float: a ph1, b ph2, rho = g/(a b) =
// 1/cos^2(theta/2) and log k = log sin(theta/2); big = 1 when rho > 8.7 (rho^32
// above 2^100) or a b = 0 (centres at or near antipodes).
struct __align__(16) XGeoRho {
    dflt ar, ai, br, bi;
    dflt rho, logk;
    int big;
    int pad[3];
};

static_assert(sizeof(XGeo) == 64 && sizeof(XGeo32) == 64 && sizeof(XGeoDF) == 64 && sizeof(XGeoRho) == 64,
              "64-byte translation records");

}  // namespace sfmm
