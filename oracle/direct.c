/*
 * oracle/direct.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * Plain, slow, obviously correct FP64 direct sum of the spherical Green's
 * function and its covariant gradient.  Only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the solver never does.
 * It shares no code with the CUDA path.
 *
 * What it computes (paper Sec. 3.1, Eq. SUM; Sec. 2.1, Eqs. GRE_FUN, ALP_PSI):
 *
 *   psi(x_i)   = sum_j q_j G(x_i, y_j),
 *   G(x, y)    = (1/4pi) [ log(1 - x.y) - log 2 ]  =  (1/4pi) log(d^2 / 4),
 *                with d^2 = |x - y|^2 = 2 (1 - x.y) for unit vectors;
 *   alpha(x_i) = covariant gradient of psi at x_i
 *              = sum_j q_j P_x (x - y_j) / (2 pi d_j^2),   P_x = I - x x^T,
 *                and P_x (x - y) = (x - y) - (d^2 / 2) x.
 *
 * d^2 is formed from the coordinate differences, never as 2(1 - x.y): the
 * latter cancels catastrophically for close pairs.  A pair with d^2 == 0
 * exactly (a target on a source, in particular a point and itself) is
 * skipped and counted; this is also how self-interaction is excluded when
 * the targets are the sources.
 *
 * alpha is returned as the tangent 3-vector and/or as its components on the
 * global basis (e_theta, e_phi) at the target, with e_theta =
 * (cos t cos p, cos t sin p, -sin t), e_phi = (-sin p, cos p, 0) and the pole
 * convention phi = atan2(0, 0) = 0.
 *
 * Every sum is Neumaier-compensated (the running sum plus a running
 * correction); OpenMP parallelises over targets only, so the result does not
 * depend on the thread count.
 */
#define _GNU_SOURCE
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stddef.h>

typedef struct { double s, c; } nsum;

static inline void nadd(nsum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                       a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum* a) { return a->s + a->c; }

/* Direct sum over all sources for targets [0, M).  Any output may be NULL.
 * psi[M], alpha2[M][2] (e_theta, e_phi), alpha3[M][3] (tangent 3-vector).
 * Returns the number of skipped coincident (d^2 == 0) pairs. */
int64_t oracle_direct(const double* src, const double* q, int64_t N,
                      const double* tgt, int64_t M,
                      double* psi, double* alpha2, double* alpha3)
{
    const double inv4pi = 1.0 / (4.0 * M_PI);
    const double inv2pi = 1.0 / (2.0 * M_PI);
    int64_t skipped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:skipped)
    for (int64_t i = 0; i < M; ++i) {
        const double x0 = tgt[3 * i], x1 = tgt[3 * i + 1], x2 = tgt[3 * i + 2];
        nsum sp = {0, 0}, g0 = {0, 0}, g1 = {0, 0}, g2 = {0, 0};
        for (int64_t j = 0; j < N; ++j) {
            const double e0 = x0 - src[3 * j];
            const double e1 = x1 - src[3 * j + 1];
            const double e2 = x2 - src[3 * j + 2];
            const double d2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (d2 == 0.0) { ++skipped; continue; }
            const double qj = q[j];
            nadd(&sp, qj * inv4pi * log(0.25 * d2));
            /* P_x (x - y) / d^2 = (x - y)/d^2 - x/2 */
            const double w = qj * inv2pi / d2;
            nadd(&g0, w * e0 - 0.5 * qj * inv2pi * x0);
            nadd(&g1, w * e1 - 0.5 * qj * inv2pi * x1);
            nadd(&g2, w * e2 - 0.5 * qj * inv2pi * x2);
        }
        const double a0 = nval(&g0), a1 = nval(&g1), a2 = nval(&g2);
        if (psi) psi[i] = nval(&sp);
        if (alpha3) { alpha3[3 * i] = a0; alpha3[3 * i + 1] = a1; alpha3[3 * i + 2] = a2; }
        if (alpha2) {
            const double rho = sqrt(x0 * x0 + x1 * x1);
            double cp = 1.0, sp_ = 0.0;           /* phi = atan2(0,0) = 0 at the poles */
            if (rho > 0.0) { cp = x0 / rho; sp_ = x1 / rho; }
            const double ct = x2, st = rho;
            const double eth0 = ct * cp, eth1 = ct * sp_, eth2 = -st;
            const double eph0 = -sp_, eph1 = cp;
            alpha2[2 * i]     = a0 * eth0 + a1 * eth1 + a2 * eth2;
            alpha2[2 * i + 1] = a0 * eph0 + a1 * eph1;
        }
    }
    return skipped;
}

/* Near Particle Model (Sec. 3.2 and Sec. 4.2, Eq. KERNEL): each mass spread
 * over a cap of angular radius sigma with the generalised Epanechnikov
 * profile W = [1 - sin^2(t/2)/sin^2(sigma/2)] / (2 pi sin^2(sigma/2)).
 * With u = sin^2(t/2) = d^2/4 and s = sin^2(sigma/2), the enclosed fraction
 * of the mass within angle t is m(u) = 2u/s - u^2/s^2 (u <= s; 1 beyond), and
 * Gauss's law on the sphere with the uniform background of Delta G = delta -
 * 1/4pi gives the deflection away from the mass
 *   2 pi sin t alpha = q (m(u) - u),  i.e. f(u) = (m - u)/(1 - u) times the
 * point-mass term q P_x(x - y)/(2 pi d^2).  The potential continues the point
 * mass's (1/4pi) log u inside the cap with the same derivative:
 *   G_s(u) = (1/4pi) [ log s + (u - s)/s^2 + ((1 - s)^2/s^2) log((1 - u)/(1 - s)) ]
 *          = (1/4pi) [ log s - (1 - u/s) + ((1 - s)^2/s^2) (log1p(t) - t) ],
 *   t = (s - u)/(1 - s)   (the second form avoids the cancellation of the two
 *   O(1/s) terms of the first),
 * so outside the cap each mass is exactly a point mass (what the far field
 * assumes).  sigma = 0 is the point-mass sum.  Pairs with d^2 == 0 are
 * skipped, as in oracle_direct. */
int64_t oracle_direct_npm(const double* src, const double* q, int64_t N,
                          const double* tgt, int64_t M, double sigma,
                          double* psi, double* alpha2, double* alpha3)
{
    const double inv4pi = 1.0 / (4.0 * M_PI);
    const double inv2pi = 1.0 / (2.0 * M_PI);
    const double sh = sin(0.5 * sigma), s = sh * sh;
    int64_t skipped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:skipped)
    for (int64_t i = 0; i < M; ++i) {
        const double x0 = tgt[3 * i], x1 = tgt[3 * i + 1], x2 = tgt[3 * i + 2];
        nsum sp = {0, 0}, g0 = {0, 0}, g1 = {0, 0}, g2 = {0, 0};
        for (int64_t j = 0; j < N; ++j) {
            const double e0 = x0 - src[3 * j];
            const double e1 = x1 - src[3 * j + 1];
            const double e2 = x2 - src[3 * j + 2];
            const double d2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (d2 == 0.0) { ++skipped; continue; }
            const double qj = q[j];
            const double u = 0.25 * d2;
            double gval, f;
            if (sigma > 0.0 && u < s) {
                const double m = 2.0 * u / s - u * u / (s * s);
                f = (m - u) / (1.0 - u);
                const double t = (s - u) / (1.0 - s);
                gval = log(s) - (1.0 - u / s) + (1.0 - s) * (1.0 - s) / (s * s) * (log1p(t) - t);
            } else {
                f = 1.0;
                gval = log(u);
            }
            nadd(&sp, qj * inv4pi * gval);
            const double w = f * qj * inv2pi / d2;
            nadd(&g0, w * e0 - 0.5 * f * qj * inv2pi * x0);
            nadd(&g1, w * e1 - 0.5 * f * qj * inv2pi * x1);
            nadd(&g2, w * e2 - 0.5 * f * qj * inv2pi * x2);
        }
        const double a0 = nval(&g0), a1 = nval(&g1), a2 = nval(&g2);
        if (psi) psi[i] = nval(&sp);
        if (alpha3) { alpha3[3 * i] = a0; alpha3[3 * i + 1] = a1; alpha3[3 * i + 2] = a2; }
        if (alpha2) {
            const double rho = sqrt(x0 * x0 + x1 * x1);
            double cp = 1.0, sp_ = 0.0;
            if (rho > 0.0) { cp = x0 / rho; sp_ = x1 / rho; }
            alpha2[2 * i] = a0 * (x2 * cp) + a1 * (x2 * sp_) - a2 * rho;
            alpha2[2 * i + 1] = -a0 * sp_ + a1 * cp;
        }
    }
    return skipped;
}

/* Potential and covariant gradient, at the points y[N], of charges h[M] and
 * tangent dipoles g[M][3] (g_i . x_i = 0) placed at the points x[M]:
 *
 *   Phi(y)       = sum_i h_i G(x_i, y) + g_i . grad_x G(x_i, y)
 *                = sum_i h_i (1/4pi) log(r^2/4) + g_i . (x_i - y) / (2 pi r^2),
 *   grad_S Phi   = P_y sum_i [ h_i (y - x_i) / (2 pi r^2)
 *                              + ( -g_i / r^2 + 2 (g_i . (x_i - y)) (x_i - y) / r^4 ) / (2 pi) ],
 *
 * r^2 = |x_i - y|^2.  The dipole term is the derivative of the point-mass
 * potential (Eq. GRE_FUN) with respect to the mass position along g_i, and
 * grad_x G = P_x (x - y)/(2 pi r^2) reduces to (x - y)/(2 pi r^2) on g_i
 * because g_i is tangent at x_i.  It is what the gradient of a loss of psi and
 * alpha with respect to the masses and their positions needs (the adjoint
 * problem).  Pairs with r^2 == 0 are skipped.  Either output may be NULL;
 * grad3 is the tangent 3-vector at y.  Returns the skipped pairs. */
int64_t oracle_dipole(const double* x, const double* h, const double* g, int64_t M,
                      const double* y, int64_t N, double* phi, double* grad3)
{
    const double inv4pi = 1.0 / (4.0 * M_PI);
    const double inv2pi = 1.0 / (2.0 * M_PI);
    int64_t skipped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:skipped)
    for (int64_t j = 0; j < N; ++j) {
        const double y0 = y[3 * j], y1 = y[3 * j + 1], y2 = y[3 * j + 2];
        nsum sp = {0, 0}, v0 = {0, 0}, v1 = {0, 0}, v2 = {0, 0};
        for (int64_t i = 0; i < M; ++i) {
            /* e = x_i - y */
            const double e0 = x[3 * i] - y0, e1 = x[3 * i + 1] - y1, e2 = x[3 * i + 2] - y2;
            const double r2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (r2 == 0.0) { ++skipped; continue; }
            const double hi = h ? h[i] : 0.0;
            const double g0 = g ? g[3 * i] : 0.0, g1 = g ? g[3 * i + 1] : 0.0, g2 = g ? g[3 * i + 2] : 0.0;
            const double ge = g0 * e0 + g1 * e1 + g2 * e2;
            nadd(&sp, hi * inv4pi * log(0.25 * r2) + ge * inv2pi / r2);
            const double wm = -hi * inv2pi / r2;              /* h (y - x) / (2 pi r^2) = -h e / (2 pi r^2) */
            const double wd = 2.0 * ge * inv2pi / (r2 * r2);
            nadd(&v0, wm * e0 - g0 * inv2pi / r2 + wd * e0);
            nadd(&v1, wm * e1 - g1 * inv2pi / r2 + wd * e1);
            nadd(&v2, wm * e2 - g2 * inv2pi / r2 + wd * e2);
        }
        if (phi) phi[j] = nval(&sp);
        if (grad3) {
            const double a0 = nval(&v0), a1 = nval(&v1), a2 = nval(&v2);
            const double yv = y0 * a0 + y1 * a1 + y2 * a2;     /* P_y v = v - (y . v) y */
            grad3[3 * j] = a0 - yv * y0;
            grad3[3 * j + 1] = a1 - yv * y1;
            grad3[3 * j + 2] = a2 - yv * y2;
        }
    }
    return skipped;
}

/* Covariant Hessian of psi = sum_j q_j G(x, y_j) at the targets, in the
 * orthonormal frame (e_theta, e_phi) (Sec. 2.2: H11 = d^2 psi/dtheta^2,
 * H12 = d/dtheta((1/sin theta) dpsi/dphi), H22 = (1/sin^2 theta) d^2 psi/dphi^2
 * + cot theta dpsi/dtheta).  For G = (1/4pi) log(1 - x.y) + const, the ambient
 * Hessian is -y y^T/(4pi (1 - x.y)^2) and the sphere adds -(x.grad G) P, so
 *   H_ab = -(e_a.d)(e_b.d)/(pi d^4) + (1 - d^2/2) delta_ab/(2 pi d^2),
 * d = x - y (e_a.y = -e_a.d because e_a is tangent at x; 1 - x.y = d^2/2).
 * hess[M][3] = (H_theta_theta, H_phi_phi, H_theta_phi).  Pairs with d^2 == 0
 * are skipped.  Returns the skipped pairs. */
int64_t oracle_hessian(const double* src, const double* q, int64_t N,
                       const double* tgt, int64_t M, double* hess)
{
    const double invpi = 1.0 / M_PI;
    int64_t skipped = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:skipped)
    for (int64_t i = 0; i < M; ++i) {
        const double x0 = tgt[3 * i], x1 = tgt[3 * i + 1], x2 = tgt[3 * i + 2];
        const double rho = sqrt(x0 * x0 + x1 * x1);
        double cp = 1.0, sp_ = 0.0;
        if (rho > 0.0) { cp = x0 / rho; sp_ = x1 / rho; }
        const double t0 = x2 * cp, t1 = x2 * sp_, t2 = -rho;      /* e_theta */
        const double f0 = -sp_, f1 = cp;                           /* e_phi */
        nsum htt = {0, 0}, hff = {0, 0}, htf = {0, 0};
        for (int64_t j = 0; j < N; ++j) {
            const double e0 = x0 - src[3 * j], e1 = x1 - src[3 * j + 1], e2 = x2 - src[3 * j + 2];
            const double d2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (d2 == 0.0) { ++skipped; continue; }
            const double dt = t0 * e0 + t1 * e1 + t2 * e2, df = f0 * e0 + f1 * e1;
            const double iso = q[j] * (1.0 - 0.5 * d2) * 0.5 * invpi / d2;
            const double w4 = q[j] * invpi / (d2 * d2);
            nadd(&htt, iso - w4 * dt * dt);
            nadd(&hff, iso - w4 * df * df);
            nadd(&htf, -w4 * dt * df);
        }
        hess[3 * i] = nval(&htt);
        hess[3 * i + 1] = nval(&hff);
        hess[3 * i + 2] = nval(&htf);
    }
    return skipped;
}

/* Number of OpenMP threads the direct sum will use (for reporting). */
int oracle_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
            n = omp_get_num_threads();
        }
    }
    return n;
}
