/*
 * sfmm.h -- C ABI of the GB300 spherical Fast Multipole Method (sFMM).
 *
 * The solver maps N point masses q_j at unit vectors y_j on the sphere S^2 to
 * the lensing potential and its covariant gradient (the deflection) at M
 * target unit vectors x_i:
 *
 *   psi(x_i)   = sum_j q_j G(x_i, y_j),                       Sec. 3.1, Eq. SUM
 *   G(x, y)    = (1/2pi) log sin(Theta/2)
 *              = (1/4pi) [log(1 - x.y) - log 2],              Sec. 2.1, Eq. GRE_FUN
 *   alpha(x_i) = covariant gradient of psi at x_i,            Sec. 2.1, Eq. ALP_PSI
 *
 * by the tree build of Sec. 3.1, the up-pass of Lemmas 1-2 (Sec. 3.1-3.2), the
 * interaction lists of Algorithm 1 with the MAC of Sec. 3.4-3.5, Lemma 3
 * (FMM-act), Lemma 4 (down-pass), the evaluation of Sec. 3.6 and the near-field
 * direct sum.  Everything runs on one CUDA device; the library never falls back
 * to the CPU.
 *
 * Conventions (apply to every entry point):
 *  - Positions are unit vectors, xyz-interleaved float64 arrays [n][3].  They
 *    are not renormalised.
 *  - alpha is returned as [M][2] float64: the components on the global basis
 *    (e_theta, e_phi) at each target, e_theta = (cos t cos p, cos t sin p,
 *    -sin t), e_phi = (-sin p, cos p, 0), with phi = atan2(0, 0) = 0 at the
 *    poles.
 *  - A source-target pair at distance exactly 0 contributes nothing (so when
 *    the targets are the sources, a point does not act on itself).
 *  - psi is the raw sum of Eq. SUM; with zero_mean set, sum_j q_j / (4 pi) is
 *    added, which makes the integral of psi over the sphere vanish (Eq.
 *    STAND_CONDITION, since the integral of G is -1).
 *  - Unless stated otherwise, array pointers are DEVICE pointers owned by the
 *    caller; the plan owns its workspace.  Work is enqueued on the plan's
 *    stream and the call returns after the result has been written (the entry
 *    points synchronise the stream once per solve to size the adaptive tree
 *    and lists).
 *  - Errors are reported as status codes, never by exceptions or device traps;
 *    sfmm_last_error() gives a message.  No kernel of this library waits on
 *    another kernel or on a flag.
 */
#ifndef SFMM_H
#define SFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfmm_plan_s* sfmm_plan_t;

typedef enum {
    SFMM_OK = 0,
    SFMM_EINVAL = 1,       /* an argument is out of range                        */
    SFMM_ENOMEM = 2,       /* a device allocation failed                         */
    SFMM_ECUDA = 3,        /* a CUDA call failed (message in sfmm_last_error)    */
    SFMM_ETIMEOUT = 4,     /* a bounded device wait gave up (its work was drained; the plan stays usable) */
    SFMM_EDEGENERATE = 5   /* reserved: degenerate input (e.g. non-finite data)  */
} sfmm_status;

enum {
    SFMM_FP64 = 0,         /* every step in float64                                                */
    SFMM_MIXED = 1,        /* stated relative error 1e-6: the near field (the bulk of the pairs) in
                              float32 on (hi, lo) offsets with compensated sums; the far field
                              (P2M, M2M, M2L, L2L, L2P) and its combination with the near field in
                              double-float (pairs of float32, about 48 bits) on the FP32 pipe      */
    SFMM_MIXED_DF = 2,     /* stated relative error 1e-10: as SFMM_MIXED with the near field in
                              double-float too                                                     */
    SFMM_FP32 = 3          /* everything in float32, M2L on the tensor cores as split-bfloat16
                              products: fastest; error about 1e-6 where the targets follow the
                              mass, but a floor of roughly eps_f32 * Q / |alpha| (up to ~1e-5)
                              on targets in smooth or empty sky, where the near and far fields
                              nearly cancel                                                        */
};

typedef struct {
    int leaf_size;         /* m of Sec. 3.1: split boxes holding more than m particles; 0 = default 32 */
    double c_s;            /* MAC1 constant of Sec. 3.5 (d - R_T - c_s R_S > 0); 0 = default 2.0 */
    double c_t;            /* MAC2 constant of Sec. 3.5 (R_T < c_t d);            0 = default 0.5 */
    int precision;         /* SFMM_FP64, SFMM_MIXED or SFMM_MIXED_DF                              */
    int zero_mean;         /* 1: add sum(q)/(4 pi) to psi (Eq. STAND_CONDITION)                    */
    int q_f32;             /* 1: the mass array is float32 instead of float64                      */
    int64_t n_max, m_max;  /* optional: size the workspace for up to n_max sources and m_max targets
                              at plan time (0 = grow on first use)                                  */
    void* stream;          /* cudaStream_t to enqueue on; NULL = the legacy default stream          */
    int m2l_tensor_cores;  /* SFMM_FP32 only: 1 (default) = M2L as split-BF16 tcgen05 GEMMs, 0 = FP32 warp kernel */
    double sigma;          /* Near Particle Model (Secs. 3.2, 4.2): each mass spread over a cap of angular
                              radius sigma with the Epanechnikov profile of Eq. KERNEL; 0 (default) = point
                              masses.  Inside the cap alpha follows from Gauss's law on the sphere
                              (f(u) = (m(u) - u)/(1 - u) times the point-mass term, u = sin^2(t/2),
                              m = 2u/s - u^2/s^2, s = sin^2(sigma/2)) and psi continues the point-mass
                              potential; far pairs also need d - R_T - R_S > sigma.  SFMM_FP64 only. */
    int wait_limit;        /* polls after which a bounded device wait (the tensor-core M2L's mbarrier waits)
                              gives up, returning SFMM_ETIMEOUT with the device context intact; 0 (default) =
                              2^26.  A test hook: a small value makes the time-out path run. */
} sfmm_options;

/* Fill *opt with the defaults listed above.  Returns SFMM_EINVAL if opt is NULL. */
sfmm_status sfmm_default_options(sfmm_options* opt);

/*
 * Create a plan (Sec. 3.7, "overview").
 *   max_depth : deepest tree level, 0..29 (r_max of Sec. 3.1; default there 29).
 *   order_p   : truncation order p of the expansions (Eq. MUL_ERR), 1..32; 0 = derive p from tol.
 *   tol       : target relative error, used only when order_p == 0 (must then be in (0, 1)).
 *   opt       : options, or NULL for the defaults.
 * On success *out holds a new plan; release it with sfmm_destroy.
 */
sfmm_status sfmm_plan(sfmm_plan_t* out, int max_depth, int order_p, double tol, const sfmm_options* opt);

/*
 * Potential only (Eq. SUM).  src_xyz [N][3], q [N] (float64, or float32 when
 * opt.q_f32), tgt_xyz [M][3] and psi [M] are device pointers; psi is
 * overwritten.  N == 0 or M == 0 is valid (psi is zero-filled).
 * SFMM_EINVAL if a pointer needed for a non-empty problem is NULL, N or M is
 * negative or exceeds 2^31 - 1.
 */
sfmm_status sfmm_potential(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                           const double* tgt_xyz, int64_t M, double* psi);

/*
 * Potential and deflection (Eqs. SUM and ALP_PSI).  As sfmm_potential, with
 * alpha [M][2] (device, overwritten).  psi may be NULL, in which case the
 * potential is not formed (the near field then needs no logarithm).
 */
sfmm_status sfmm_deflection(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                            const double* tgt_xyz, int64_t M, double* psi, double* alpha);

/*
 * sfmm_deflection with HOST arrays: the inputs are copied to the plan's device
 * workspace and the results copied back inside the call (pinned host memory
 * gives the fastest copies; pageable memory also works).  psi may be NULL.
 */
sfmm_status sfmm_deflection_host(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                                 const double* tgt_xyz, int64_t M, double* psi, double* alpha);

/*
 * Batched shells (the multi-layer setting of Sec. 2.1: N_L independent
 * lensing planes): shell i has its own sources src_xyz[i] [N[i]][3], masses
 * q[i] and targets tgt_xyz[i] [M[i]][3]; results go to psi[i] (or psi == NULL
 * / psi[i] == NULL for none) and alpha[i] [M[i]][2].  All pointers inside
 * the arrays are device pointers; the arrays themselves are host arrays of
 * n_shells entries.  The shells are solved with the plan's settings by
 * `lanes` (1..8) internal solvers, each on its own stream driven by its own
 * host thread, largest shells first, so that one shell's latency-bound
 * phases (tree levels, list walk) overlap the kernels of another.  Work
 * queued earlier on the plan's stream happens before, and work queued later
 * after, all shells.  Each lane keeps a workspace sized for the largest shell
 * it met.  On failure the first failing shell's status is returned.
 */
sfmm_status sfmm_deflection_batch(sfmm_plan_t plan, int n_shells, const double* const* src_xyz,
                                  const void* const* q, const int64_t* N, const double* const* tgt_xyz,
                                  const int64_t* M, double* const* psi, double* const* alpha, int lanes);

/*
 * Graph-launched shells (the N_L lensing planes of Sec. 2.1, as for
 * sfmm_deflection_batch, replayed as one CUDA graph).
 *
 * sfmm_graph_capture binds the plan to a batch of shells: the same arrays as
 * sfmm_deflection_batch (device pointers in host arrays of n_shells entries;
 * psi may be NULL).  It solves every shell once, synchronously (the results
 * are valid on return), plans each shell's capacities (nodes, level width,
 * levels, M2L and P2P pairs) as its counts times (1 + slack) plus a margin
 * (slack in [0, 16]; 0 selects 0.25), and records the solves of all shells,
 * with no host synchronisation inside, into one CUDA graph: each shell on its
 * own stream and workspace, its tree, lists and launches sized by its
 * capacities and its counts read on the device.  The sizes N[i], M[i] and the
 * buffers are fixed by the capture; their CONTENTS may change between
 * launches (new positions and masses).  The caller keeps the buffers alive
 * until sfmm_graph_release or sfmm_destroy.  Plans of precision SFMM_FP64,
 * SFMM_MIXED or SFMM_MIXED_DF with point masses (sigma == 0); SFMM_EINVAL
 * otherwise.  A previous capture is released.
 *
 * sfmm_graph_launch replays the graph on the plan's stream and waits for it
 * (one synchronisation for all shells).  A shell whose new data outgrew a
 * capacity (a deeper or wider tree, more pairs) is detected on the device; it
 * is solved again synchronously, so the results are valid on return, and the
 * graph is recorded again with capacities planned from the new data.
 *
 * sfmm_graph_info reports the graph (zeros when there is none): kernel nodes
 * per replay, replays, overflowed shells, re-recordings and the summed counts
 * of the last replay.  sfmm_graph_release frees the graph and its workspaces.
 */
typedef struct {
    int64_t n_shells;
    int64_t kernel_nodes;   /* kernels launched by one replay */
    int64_t launches, overflows, recaptures;
    int64_t n_nodes, n_leaves, n_m2l, n_p2p;   /* summed over the shells, last replay */
} sfmm_graph_stats;

sfmm_status sfmm_graph_capture(sfmm_plan_t plan, int n_shells, const double* const* src_xyz, const void* const* q,
                               const int64_t* N, const double* const* tgt_xyz, const int64_t* M, double* const* psi,
                               double* const* alpha, double slack);
sfmm_status sfmm_graph_launch(sfmm_plan_t plan);
sfmm_status sfmm_graph_info(sfmm_plan_t plan, sfmm_graph_stats* out);
sfmm_status sfmm_graph_release(sfmm_plan_t plan);

/*
 * Shear and magnification (Sec. 2.2, Eq. GAM_DEF): gamma [M][2] = (gamma_1,
 * gamma_2), the trace-free part of the covariant Hessian H of psi on
 * (e_theta, e_phi) at each target, gamma_1 = (H11 - H22)/2, gamma_2 = H12, and
 * (if mu is not NULL) mu [M] = 1/((1 - tr H/2)^2 - gamma_1^2 - gamma_2^2), the
 * magnification of a small source (Sec. 2.2).  For point masses the trace is
 * kappa - kappa_bar = tr H = -sum(q)/(4 pi) at a target off the masses
 * (Delta G = delta - 1/(4 pi)); a target on a mass skips that mass, in the
 * trace as in every output.  psi and alpha as in sfmm_deflection (either may
 * be NULL).  Far field from the second derivative of each leaf's local
 * expansion (conformal chart), near field from the closed form of the Hessian
 * of G.  Runs in FP64 whatever opt.precision is.
 */
sfmm_status sfmm_shear(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                       const double* tgt_xyz, int64_t M, double* psi, double* alpha, double* gamma, double* mu);

/*
 * Adjoint: gradients of a loss L(psi, alpha) of sfmm_deflection's outputs with
 * respect to the masses and the source positions, given dL/dpsi and
 * dL/dalpha at the targets.  With g_i = g_alpha[i][0] e_theta(x_i) +
 * g_alpha[i][1] e_phi(x_i) (the basis alpha is written in) and
 * Phi(y) = sum_i g_psi[i] G(x_i, y) + g_i . grad_x G(x_i, y):
 *   grad_q[j]   = dL/dq_j = Phi(y_j)   (+ sum_i g_psi[i] / 4pi with opt.zero_mean),
 *   grad_src[j] = dL/dy_j = q_j grad_S Phi(y_j), the covariant (tangent)
 *                 gradient on the sphere as a 3-vector [N][3].
 * This is one more sFMM: charges g_psi and tangent dipoles g at the targets
 * (the dipole multipole is Lemma 1 differentiated along g), evaluated at the
 * sources; M2M, M2L and L2L are those of the forward solve.  With the plan's
 * p, leaf size and MAC, it runs in FP64 for an SFMM_FP64 plan and otherwise in
 * double-float (the far field of SFMM_MIXED_DF, a double-float near field of
 * charges and dipoles; about 1e-12 relative).  Arguments
 * as for sfmm_deflection (device pointers; q float32 when opt.q_f32); g_psi
 * [M] and g_alpha [M][2] may be NULL (treated as zero); at least one of
 * grad_q [N], grad_src [N][3] must be non-NULL.  Gradients with respect to the
 * target positions are not formed.  The paper has no adjoint; this follows
 * from Eqs. SUM, GRE_FUN and ALP_PSI by linearity in q and symmetry of G.
 */
sfmm_status sfmm_adjoint(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                         const double* tgt_xyz, int64_t M, const double* g_psi, const double* g_alpha,
                         double* grad_q, double* grad_src);

/* Release the plan and its workspace.  NULL is ignored. */
void sfmm_destroy(sfmm_plan_t plan);

/* Message for the last failing call on this plan ("" if none).  The string
 * is owned by the plan.  With plan == NULL, the message of the last failed
 * sfmm_plan() call of this process. */
const char* sfmm_last_error(sfmm_plan_t plan);

/* The order p in use (resolved from tol when the plan was made with order_p == 0). */
int sfmm_order(sfmm_plan_t plan);

/*
 * Statistics of the last solve on this plan (host struct, filled by copy).
 *   n_nodes, n_leaves, depth : the tree of Sec. 3.1 (depth = deepest level used)
 *   n_m2l, n_p2p             : FMM-act and direct-act pairs of Algorithm 1
 *   p2p_interactions         : source-target point pairs evaluated directly (counted
 *                              only while timing is at level 2, else 0)
 *   launches                 : kernel launches of the solve
 *   ms[8]                    : device time of the phases on the plan's stream (only
 *                              while timing is on): keys+sort, tree+geometry, up-pass,
 *                              lists, M2L, L2L, evaluation, total
 *   near_ms                  : SFMM_MIXED: device time of the near-field kernel, which
 *                              runs on the auxiliary stream beside M2L and L2L (its
 *                              evaluation phase is then the double-float finish); else 0
 */
typedef struct {
    int64_t n_nodes, n_leaves, depth, n_m2l, n_p2p, p2p_interactions, launches;
    double ms[8];
    double near_ms;
} sfmm_stats;
sfmm_status sfmm_get_stats(sfmm_plan_t plan, sfmm_stats* out);

/* Change the plan's wait_limit (sfmm_options.wait_limit) for later solves: 0 = the default
 * bound; a small value makes the bounded device waits run out (a test hook).  SFMM_EINVAL
 * for a negative value. */
sfmm_status sfmm_set_wait_limit(sfmm_plan_t plan, int polls);

/* Record per-phase device times (CUDA events) in later solves: 0 off (default), 1 phase
 * times, 2 phase times and the count of near-field point pairs (one more kernel and a
 * host synchronisation per solve, inside the evaluation phase's time). */
sfmm_status sfmm_set_timing(sfmm_plan_t plan, int on);

/*
 * Introspection for tests: copy an internal array of the last solve to HOST
 * memory `dst` of `bytes` bytes (the exact size is returned in *bytes_needed
 * when dst is NULL).  Arrays (node arrays are in tree order: by level, then by
 * pixel index; particles in key order):
 *   SFMM_ARR_SRC_KEYS      uint64 [N]      sorted order-29 nested keys of the sources
 *   SFMM_ARR_SRC_PERM      int32  [N]      original index of each sorted source
 *   SFMM_ARR_NODE_PREFIX   uint64 [nodes]  nested pixel index of each box at its level
 *   SFMM_ARR_NODE_LEVEL    int32  [nodes]
 *   SFMM_ARR_NODE_RANGE    int32  [nodes][2]  first, count in the sorted sources
 *   SFMM_ARR_NODE_CHILD0   int32  [nodes]  first child (children are consecutive) or -1
 *   SFMM_ARR_NODE_PARENT   int32  [nodes]  parent or -1 for a base box
 *   SFMM_ARR_NODE_GEOM     double [nodes][11]  centre xyz, e_theta xyz, e_phi xyz, R, tan(R/2)
 *   SFMM_ARR_MULTIPOLE     double [nodes][2p+2] C, Q, Re A_1, Im A_1, ... (unscaled, frame K_P)
 *   SFMM_ARR_LOCAL         double [nodes][2p+2] C, Q, Re A_1, Im A_1, ... (unscaled, frame K_P)
 *   SFMM_ARR_M2L           int32  [n_m2l][2]  (source, target) pairs grouped by target
 *   SFMM_ARR_P2P           int32  [n_p2p][2]  (source leaf, target leaf) grouped by target
 *   SFMM_ARR_TGT_KEYS      uint64 [M]      sorted keys of the targets
 *   SFMM_ARR_NODE_TRANGE   int32  [nodes][2]  first, count in the sorted targets
 *   SFMM_ARR_SRC_OFFSETS   float  [N][8]   (every format but SFMM_FP64; else 0 bytes) per sorted
 *                                          source: hi x, y, z, q, then lo x, y, z, q of its offset from
 *                                          its leaf's centre and of its mass (value = hi + lo)
 *   SFMM_ARR_TGT_OFFSETS   float  [M][8]   (as above) per sorted target: hi x, y, z, 0, lo x, y, z, 0
 */
enum {
    SFMM_ARR_SRC_KEYS = 0, SFMM_ARR_SRC_PERM, SFMM_ARR_NODE_PREFIX, SFMM_ARR_NODE_LEVEL,
    SFMM_ARR_NODE_RANGE, SFMM_ARR_NODE_CHILD0, SFMM_ARR_NODE_PARENT, SFMM_ARR_NODE_GEOM,
    SFMM_ARR_MULTIPOLE, SFMM_ARR_LOCAL, SFMM_ARR_M2L, SFMM_ARR_P2P, SFMM_ARR_TGT_KEYS,
    SFMM_ARR_NODE_TRANGE, SFMM_ARR_SRC_OFFSETS, SFMM_ARR_TGT_OFFSETS
};
sfmm_status sfmm_debug_copy(sfmm_plan_t plan, int which, void* dst, int64_t bytes, int64_t* bytes_needed);

/*
 * The order-29 nested HEALPix key (Sec. 3.1; Gorski et al. 2005) of n unit
 * vectors xyz [n][3] (device) into keys [n] (device, uint64), enqueued on
 * `stream` (cudaStream_t or NULL).  The same routine the tree build uses.
 */
sfmm_status sfmm_keys(const double* xyz, int64_t n, uint64_t* keys, void* stream);

/*
 * The keys and stable radix sort of sfmm_keys / the first step of every solve,
 * for callers that must not allocate device memory (a plugin inside a host
 * application whose memory pool owns the device, a latency-critical pipeline
 * that cannot accept the synchronisation cudaMalloc/cudaFree may cause).  The
 * paper has no counterpart; this is a property of the library, not of the method.
 *   xyz   [n][3] float64 unit vectors (device, caller-owned)
 *   keys  [n] uint64 (device, caller-owned, overwritten): the order-29 nested keys
 *         in ascending order
 *   perm  [n] uint32 (device, caller-owned, overwritten): perm[i] = input index of
 *         the i-th smallest key; equal keys keep their input order
 *   n     0..262144: larger n returns SFMM_EINVAL (message in sfmm_last_error(NULL))
 * Allocates nothing: the sort's scratch (3.5 MiB) is one static device array
 * that every GPU loading the library holds until exit.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and should
 * come before any stream capture.  All calls share the array: calls that
 * overlap on the GPU race and must be serialised by the caller.  Work is
 * enqueued on `stream` (cudaStream_t or NULL); the outputs are ready when the
 * stream reaches that point.
 */
sfmm_status sfmm_sort_keys_static(const double* xyz, int64_t n, uint64_t* keys, uint32_t* perm, void* stream);

/*
 * Measured arithmetic rate of this GPU (the denominators of the evaluation
 * kernels' rooflines; the paper has no counterpart): which = 0 FP32 FMA,
 * 1 packed FP32x2 FMA, 2 FP64 FMA (flop/s, an FMA counted as 2), 3 MUFU
 * reciprocal + base-2 logarithm (operations/s).  A loop of independent chains on
 * a full grid, timed with CUDA events on `stream` (cudaStream_t or NULL) after
 * a warm-up launch; about half a second each.  Allocates 16 bytes of device
 * memory for the duration of the call.  SFMM_EINVAL for another `which` or a
 * NULL ops_per_s.
 */
sfmm_status sfmm_peak_rate(int which, double* ops_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFMM_H */
