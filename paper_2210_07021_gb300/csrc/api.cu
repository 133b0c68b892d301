// The C ABI of include/sfmm.h: plan management and the solve pipeline
// (Sec. 3.7 overview): keys + sort -> tree (Sec. 3.1) -> P2M / M2M (Lemmas 1-2)
// -> interaction lists (Algorithm 1, Sec. 3.4-3.5) -> M2L (Lemma 3) -> L2L
// (Lemma 4) -> L2P + near field (Sec. 3.6).  Every step runs on the device.
#include "common.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

namespace sfmm {
cudaError_t build_tree(sfmm_plan_s* P, const uint64_t* keys, int64_t n, int m, int max_depth);
cudaError_t tree_geometry(sfmm_plan_s* P);
cudaError_t tree_target_ranges(sfmm_plan_s* P, const uint64_t* tkeys, int64_t M);
cudaError_t collect_leaves(sfmm_plan_s* P, const int* cnt, Buf& out, int64_t* n_out, int64_t* d_out);
cudaError_t build_lists(sfmm_plan_s* P, const TreeView& T, double c_s, double c_t, cudaStream_t s);
void fill_tables(double* h);
size_t xgeo_bytes(int ek);
cudaError_t launch_geom32(int n_nodes, const double* geom, float* g32, cudaStream_t s);
cudaError_t launch_pair_geo(const TreeView& T, const float* g32, const uint64_t* tt, const uint32_t* ss, int64_t n,
                            const int64_t* d_n, void* out, int ek, cudaStream_t s);
cudaError_t launch_child_geo(const TreeView& T, const float* g32, void* m2m, void* l2l, int ek, cudaStream_t s);
cudaError_t launch_src_offsets(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                               const double4_32a* src, float4* off, cudaStream_t s);
cudaError_t launch_p2m(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                       const double4_32a* src, const float4* off, const float4* log_tab, void* mpole, int p, int ek,
                       cudaStream_t s);
cudaError_t launch_m2m(const TreeView& T, int a, int b, int lvl, int p, const double* tables, const void* geo,
                       void* mpole, int ek, cudaStream_t s);
cudaError_t launch_m2l(const TreeView& T, const int64_t* off, const uint32_t* srcs, int p, const double* tables,
                       const void* geo, const void* mpole, void* local, int ek, cudaStream_t s);
cudaError_t launch_m2l_list(const uint64_t* ptgt, const uint32_t* psrc, const uint32_t* list, const uint32_t* n_list,
                            int64_t max_list, int p, const double* tables, const void* geo, const void* mpole,
                            void* local, cudaStream_t s);
cudaError_t launch_m2l_tc(int64_t n_pairs, const uint64_t* ptgt, const uint32_t* psrc, const void* geo,
                          const void* mpole, void* local, int p, uint32_t* leftover, uint32_t* n_leftover,
                          uint32_t* tile_ctr, int* status, int wait_limit, cudaStream_t s);
cudaError_t launch_l2l(const TreeView& T, int a, int b, int lvl, int p, const double* tables, const void* geo,
                       void* local, int ek, cudaStream_t s);
size_t frame_df_bytes();
cudaError_t launch_frame_df(int n_nodes, const int64_t* d_nn, const double* geom, void* out, cudaStream_t s);
cudaError_t launch_pair_geo_rho(const TreeView& T, const void* frames, const float4* log_tab, const uint64_t* tt,
                                const uint32_t* ss, int64_t n, const int64_t* d_n, void* out, cudaStream_t s);
cudaError_t launch_child_geo_df(const TreeView& T, const void* frames, const float4* log_tab, void* m2m, void* l2l,
                                cudaStream_t s);
cudaError_t launch_m2l_pair(int64_t n_pairs, const int64_t* d_n, const uint64_t* ptgt, const uint32_t* psrc, const void* geo,
                            const void* mpole, int p, double* acc, uint32_t* leftover, uint32_t* n_left,
                            cudaStream_t s);
cudaError_t launch_m2l_left_df(const TreeView& T, const uint64_t* ptgt, const uint32_t* psrc, const uint32_t* list,
                               const uint32_t* n_list, int64_t max_list, int p, const double* tables,
                               const void* mpole, double* acc, cudaStream_t s);
cudaError_t launch_acc_to_df(int64_t n, const double* acc, void* out, cudaStream_t s);
cudaError_t launch_m2m_df(const TreeView& T, int c0, int c1, int lvl, int p, const void* geo, void* mpole,
                          cudaStream_t s);
cudaError_t launch_l2l_df(const TreeView& T, int a, int b, int lvl, int p, const void* geo, const double* acc,
                          void* local, cudaStream_t s);
cudaError_t launch_p2m_df_leaf(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* off,
                               const float4* doff, const float4* log_tab, int p, void* mpole, cudaStream_t s);
cudaError_t launch_unscale(int n_nodes, const double* geom, const void* in, double* out, int p, int is_local,
                           int ek, cudaStream_t s);
cudaError_t launch_eval32_prep(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl,
                               const double4_32a* tgt, float4* toff, const uint64_t* p2p_t, const uint32_t* p2p_s,
                               int64_t n_p2p, const int64_t* d_np, float4* dc, cudaStream_t s);
cudaError_t launch_eval32(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* soff,
                          const float4* toff, const float4* dc, const double4_32a* tgt, const uint32_t* tperm, const int64_t* p2p_off,
                          const uint32_t* p2p_src, const void* local, const void* mpole, bool dfar, int p, int zero_mean,
                          double* psi, double* alpha, bool coincide, float4* nf, int* tleaf,
                          const void* frames, int64_t M, int what, unsigned long long* leaf_ctr, cudaStream_t s);
cudaError_t launch_count_pairs(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* p2p_off,
                               const uint32_t* p2p_src, unsigned long long* out, cudaStream_t s);
void fill_log_table(float* out);
cudaError_t launch_eval_df(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const float4* soff,
                           const float4* toff, const float4* dc, const double4_32a* tgt, const uint32_t* tperm,
                           const int64_t* p2p_off, const uint32_t* p2p_src, const void* local, const void* mpole,
                           const float4* log_tab, int p, int zero_mean, double* psi, double* alpha,
                           const float4* doff, const void* w, int w_f32, double* grad3, float4* nf, int* tleaf,
                           const void* frames, int64_t M, int what, unsigned long long* leaf_ctr, cudaStream_t s);
cudaError_t launch_p2m_adj(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src,
                           const double4_32a* dip, double* mpole, int p, cudaStream_t s);
cudaError_t launch_eval_adj(const TreeView& T, const int* leaves, int64_t n_leaves, const double4_32a* src,
                            const double4_32a* dip, const double4_32a* tgt, const uint32_t* tperm,
                            const int64_t* p2p_off, const uint32_t* p2p_src, const double* local, const double* mpole,
                            int p, int zero_mean, const void* w, int w_f32, double* phi, double* grad3,
                            unsigned long long* leaf_ctr, cudaStream_t s);
cudaError_t launch_eval(const TreeView& T, const int* leaves, int64_t n_leaves, const int64_t* d_nl, const double4_32a* src,
                        const double4_32a* tgt,
                        const uint32_t* tperm, const int64_t* p2p_off, const uint32_t* p2p_src, const double* local,
                        const double* mpole, int p, int zero_mean, double sigma, double* psi, double* alpha,
                        double* gamma, double* mu, unsigned long long* leaf_ctr, cudaStream_t s);

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t ensure(Buf& b, size_t bytes)
{
    if (bytes <= b.cap && b.p) return cudaSuccess;
    if (b.p) { cudaFree(b.p); b.p = nullptr; b.cap = 0; }
    size_t nb = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) { b.p = nullptr; return e; }
    b.cap = nb;
    return cudaSuccess;
}

cudaError_t ensure_keep(Buf& b, size_t bytes, size_t keep, cudaStream_t s)
{
    if (bytes <= b.cap && b.p) return cudaSuccess;
    size_t nb = bytes < 256 ? 256 : bytes;
    void* np = nullptr;
    cudaError_t e = cudaMalloc(&np, nb);
    if (e != cudaSuccess) return e;
    if (b.p && keep) {
        e = cudaMemcpyAsync(np, b.p, keep < b.cap ? keep : b.cap, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { cudaFree(np); return e; }
        cudaStreamSynchronize(s);
    }
    if (b.p) cudaFree(b.p);
    b.p = np;
    b.cap = nb;
    return cudaSuccess;
}

void release(Buf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

namespace {

std::mutex g_err_mu;
std::string g_plan_err;

__global__ void k_gather_src(const double* __restrict__ xyz, const void* __restrict__ q, int q_f32,
                             const uint32_t* __restrict__ perm, int64_t n, double4_32a* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[i];
        const double qq = q_f32 ? (double)static_cast<const float*>(q)[j] : static_cast<const double*>(q)[j];
        out[i] = make_double4_32a(xyz[3 * (size_t)j], xyz[3 * (size_t)j + 1], xyz[3 * (size_t)j + 2], qq);
    }
}

// tangent dipoles of the adjoint into key order (g_x, g_y, g_z, 0)
__global__ void k_gather_dip(const double* __restrict__ g, const uint32_t* __restrict__ perm, int64_t n,
                             double4_32a* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[i];
        out[i] = make_double4_32a(g[3 * (size_t)j], g[3 * (size_t)j + 1], g[3 * (size_t)j + 2], 0.0);
    }
}

// tangent dipoles of the adjoint into key order as (hi, lo) float4 pairs:
// out[2i] = (g_x, g_y, g_z) leading parts, out[2i + 1] their remainders
__global__ void k_gather_dip_df(const double* __restrict__ g, const uint32_t* __restrict__ perm, int64_t n,
                                float4* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[i];
        const dflt x(g[3 * (size_t)j]), y(g[3 * (size_t)j + 1]), z(g[3 * (size_t)j + 2]);
        out[2 * i] = make_float4(x.h, y.h, z.h, 0.f);
        out[2 * i + 1] = make_float4(x.l, y.l, z.l, 0.f);
    }
}

// Adjoint sources at the forward targets x_i: charge h_i = dL/dpsi_i (0 without
// one) and tangent dipole g_i = dL/dalpha_i[0] e_theta(x_i) + dL/dalpha_i[1]
// e_phi(x_i), the basis the forward path writes alpha in (phi = 0 at the poles).
__global__ void k_adjoint_prep(const double* __restrict__ x, int64_t m, const double* __restrict__ g_psi,
                               const double* __restrict__ g_alpha, double* __restrict__ h, double* __restrict__ dip)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        h[i] = g_psi ? g_psi[i] : 0.0;
        double a = 0.0, b = 0.0;
        if (g_alpha) { a = g_alpha[2 * i]; b = g_alpha[2 * i + 1]; }
        const double rho = sqrt(x0 * x0 + x1 * x1);
        double cp = 1.0, sp = 0.0;
        if (rho > 0.0) { cp = x0 / rho; sp = x1 / rho; }
        dip[3 * i] = a * (x2 * cp) - b * sp;
        dip[3 * i + 1] = a * (x2 * sp) + b * cp;
        dip[3 * i + 2] = -a * rho;
    }
}

__global__ void k_fill(double* __restrict__ p, int64_t n, double v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_gather_tgt(const double* __restrict__ xyz, const uint32_t* __restrict__ perm, int64_t n,
                             double4_32a* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = perm[i];
        out[i] = make_double4_32a(xyz[3 * (size_t)j], xyz[3 * (size_t)j + 1], xyz[3 * (size_t)j + 2], 0.0);
    }
}

inline unsigned grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

// p from a tolerance: the error of the far field falls roughly as 0.5^p under
// the default MAC; the table is refined by measurement.
int p_from_tol(double tol)
{
    int p = (int)std::ceil(std::log(tol) / std::log(0.5));
    if (p < 4) p = 4;
    if (p > PMAX) p = PMAX;
    return p;
}

sfmm_status fail(sfmm_plan_s* P, sfmm_status st, const std::string& msg)
{
    if (P) P->err = msg;
    return st;
}

sfmm_status cuda_fail(sfmm_plan_s* P, cudaError_t e, const char* where)
{
    char b[256];
    snprintf(b, sizeof b, "CUDA error in %s: %s", where, cudaGetErrorString(e));
    return fail(P, e == cudaErrorMemoryAllocation ? SFMM_ENOMEM : SFMM_ECUDA, b);
}

TreeView view(sfmm_plan_s* P)
{
    TreeView T;
    T.n_nodes = (int)P->n_nodes;
    DevCounts* dc = P->gm ? P->dcnt.as<DevCounts>() : nullptr;
    T.d_nn = dc ? &dc->nn : nullptr;
    T.d_level = dc ? dc->level : nullptr;
    T.prefix = P->n_prefix.as<uint64_t>();
    T.level = P->n_level.as<int>();
    T.first = P->n_first.as<int>();
    T.count = P->n_count.as<int>();
    T.child0 = P->n_child0.as<int>();
    T.parent = P->n_parent.as<int>();
    T.geom = P->n_geom.as<double>();
    T.tfirst = P->n_tfirst.as<int>();
    T.tcount = P->n_tcount.as<int>();
    return T;
}

struct PhaseTimer {
    sfmm_plan_s* P;
    cudaEvent_t ev[8];
    int n = 0;
    explicit PhaseTimer(sfmm_plan_s* p) : P(p)
    {
        if (P->timing)
            for (auto& e : ev) cudaEventCreate(&e);
    }
    void mark()
    {
        if (P->timing && n < 8) cudaEventRecord(ev[n++], P->stream);
    }
    void finish()
    {
        if (!P->timing) return;
        cudaEventSynchronize(ev[n - 1]);
        for (int i = 0; i + 1 < n && i < 7; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            P->stats.ms[i] = ms;
        }
        float tot = 0;
        cudaEventElapsedTime(&tot, ev[0], ev[n - 1]);
        P->stats.ms[7] = tot;
    }
    ~PhaseTimer()
    {
        if (P->timing)
            for (auto& e : ev) cudaEventDestroy(e);
    }
};

// The adjoint's extra inputs and outputs: tangent dipoles at the sources,
// weights of the targets' gradient output and that output ([M][3]).
struct AdjIO {
    const double* dip;
    const void* w;
    int w_f32;
    double* grad3;
};

sfmm_status solve(sfmm_plan_s* P, const double* src, const void* q, int64_t N, const double* tgt, int64_t M,
                  double* psi, double* alpha, const AdjIO* adj = nullptr, double* gamma = nullptr,
                  double* mu = nullptr)
{
    cudaStream_t s = P->stream;
    // the shear runs in FP64; the adjoint in FP64 for FP64 plans, else with the double-float far
    // and near fields (its own near-field kernel, charges and dipoles)
    const bool adj_df = adj && P->opt.precision != SFMM_FP64;
    const int precision = gamma ? SFMM_FP64 : adj ? (adj_df ? SFMM_MIXED_DF : SFMM_FP64) : P->opt.precision;
    if (P->gm && !(precision == SFMM_MIXED || precision == SFMM_MIXED_DF || precision == SFMM_FP64))
        return fail(P, SFMM_EINVAL, "graph mode runs SFMM_FP64, SFMM_MIXED and SFMM_MIXED_DF plans");
    const int q_f32 = adj ? 0 : P->opt.q_f32;
    cudaError_t e;
    const int p = P->p;
    P->err.clear();
    P->stats = sfmm_stats{};
    P->last_N = N;
    P->last_M = M;
    P->n_nodes = 0;
    const int64_t launches0 = launch_total();
    if (M > 0 && N == 0) {
        if (psi && (e = cudaMemsetAsync(psi, 0, (size_t)M * 8, s))) return cuda_fail(P, e, "memset psi");
        if (alpha && (e = cudaMemsetAsync(alpha, 0, (size_t)M * 16, s))) return cuda_fail(P, e, "memset alpha");
        if (adj && adj->grad3 && (e = cudaMemsetAsync(adj->grad3, 0, (size_t)M * 24, s)))
            return cuda_fail(P, e, "memset gradient");
        if (gamma && (e = cudaMemsetAsync(gamma, 0, (size_t)M * 16, s))) return cuda_fail(P, e, "memset gamma");
        if (mu) {       // no mass: H = 0, mu = 1
            k_fill<<<grid_for(M), 256, 0, s>>>(mu, M, 1.0); count_launch();
            if ((e = cudaGetLastError())) return cuda_fail(P, e, "mu");
        }
        if (!P->gm && (e = cudaStreamSynchronize(s))) return cuda_fail(P, e, "sync");
        return SFMM_OK;
    }
    if (M == 0) return SFMM_OK;
    // graph mode: the counts live in the plan's DevCounts (see build_tree); launches
    // over leaves and pairs are sized by capacities and read the counts there
    DevCounts* dcnt = P->gm ? P->dcnt.as<DevCounts>() : nullptr;
    PhaseTimer tm(P);
    tm.mark();
    // ---- keys and sort (sources and targets)
    if ((e = ensure(P->small, 64 * 8))) return cuda_fail(P, e, "alloc");
    if ((e = ensure(P->skeys, N * 8)) || (e = ensure(P->skeys2, N * 8)) || (e = ensure(P->sperm, N * 4)) ||
        (e = ensure(P->sperm2, N * 4)) || (e = ensure(P->src4, N * 32)))
        return cuda_fail(P, e, "alloc sources");
    if ((e = ensure(P->tkeys, M * 8)) || (e = ensure(P->tkeys2, M * 8)) || (e = ensure(P->tperm, M * 4)) ||
        (e = ensure(P->tperm2, M * 4)) || (e = ensure(P->tgt4, M * 32)))
        return cuda_fail(P, e, "alloc targets");
    if ((e = ensure(P->tmp, radix_tmp_bytes(std::max(N, M)))) || (e = ensure(P->ttmp, radix_tmp_bytes(M))))
        return cuda_fail(P, e, "alloc");
    // The targets' keys, sort and gather need nothing from the sources: they run
    // on the auxiliary stream (forked from and joined back into the plan's
    // stream by events, with their own sort scratch) while the plan's stream
    // sorts the sources, builds the tree (one host synchronisation per level)
    // and runs the up-pass.
    cudaStream_t s2 = P->aux;
    if (P->forked) P->forked = false;
    else if ((e = cudaEventRecord(P->ev_fork, s)) || (e = cudaStreamWaitEvent(s2, P->ev_fork, 0)))
        return cuda_fail(P, e, "fork");
    if ((e = launch_keys(tgt, M, P->tkeys.as<uint64_t>(), P->tperm.as<uint32_t>(), s2))) return cuda_fail(P, e, "tkeys");
    if ((e = radix_sort(P->tkeys.as<uint64_t>(), P->tperm.as<uint32_t>(), P->tkeys2.as<uint64_t>(),
                        P->tperm2.as<uint32_t>(), M, 62, P->ttmp.p, s2, &P->tkeys_alt)))
        return cuda_fail(P, e, "sort targets");
    const uint64_t* tkeys = P->tkeys_alt ? P->tkeys2.as<uint64_t>() : P->tkeys.as<uint64_t>();
    const uint32_t* tperm = P->tkeys_alt ? P->tperm2.as<uint32_t>() : P->tperm.as<uint32_t>();
    k_gather_tgt<<<grid_for(M), 256, 0, s2>>>(tgt, tperm, M, P->tgt4.as<double4_32a>()); count_launch();
    if ((e = cudaGetLastError()) || (e = cudaEventRecord(P->ev_join, s2))) return cuda_fail(P, e, "gather targets");
    if ((e = launch_keys(src, N, P->skeys.as<uint64_t>(), P->sperm.as<uint32_t>(), s))) return cuda_fail(P, e, "keys");
    if ((e = radix_sort(P->skeys.as<uint64_t>(), P->sperm.as<uint32_t>(), P->skeys2.as<uint64_t>(),
                        P->sperm2.as<uint32_t>(), N, 62, P->tmp.p, s, &P->skeys_alt)))
        return cuda_fail(P, e, "sort sources");
    const uint64_t* skeys = P->skeys_alt ? P->skeys2.as<uint64_t>() : P->skeys.as<uint64_t>();
    const uint32_t* sperm = P->skeys_alt ? P->sperm2.as<uint32_t>() : P->sperm.as<uint32_t>();
    k_gather_src<<<grid_for(N), 256, 0, s>>>(src, q, q_f32, sperm, N, P->src4.as<double4_32a>()); count_launch();
    if (adj_df) {
        if ((e = ensure(P->dip4, (size_t)N * 32))) return cuda_fail(P, e, "alloc dipoles");
        k_gather_dip_df<<<grid_for(N), 256, 0, s>>>(adj->dip, sperm, N, P->dip4.as<float4>()); count_launch();
    } else if (adj) {
        if ((e = ensure(P->dip4, (size_t)N * 32))) return cuda_fail(P, e, "alloc dipoles");
        k_gather_dip<<<grid_for(N), 256, 0, s>>>(adj->dip, sperm, N, P->dip4.as<double4_32a>()); count_launch();
    }
    if ((e = cudaGetLastError())) return cuda_fail(P, e, "gather");
    tm.mark();
    // ---- tree and geometry (sources)
    if ((e = build_tree(P, skeys, N, P->opt.leaf_size, P->max_depth))) return cuda_fail(P, e, "tree");
    const int64_t nn = P->n_nodes;
    if ((e = tree_geometry(P))) return cuda_fail(P, e, "geometry");
    TreeView T = view(P);
    if ((e = collect_leaves(P, T.count, P->leaves_src, &P->n_leaves, dcnt ? &dcnt->n_leaves : nullptr)))
        return cuda_fail(P, e, "leaves");
    const int64_t* d_nls = dcnt ? &dcnt->n_leaves : nullptr;
    const int64_t* d_nlt = dcnt ? &dcnt->n_leaves_tgt : nullptr;
    tm.mark();
    // ---- join the targets; target ranges (Sec. 3.7 lookup) and target leaves
    if ((e = cudaStreamWaitEvent(s, P->ev_join, 0))) return cuda_fail(P, e, "join");
    if ((e = tree_target_ranges(P, tkeys, M))) return cuda_fail(P, e, "target ranges");
    T = view(P);
    if ((e = collect_leaves(P, T.tcount, P->leaves_tgt, &P->n_leaves_tgt, dcnt ? &dcnt->n_leaves_tgt : nullptr)))
        return cuda_fail(P, e, "target leaves");
    // ---- up-pass on the plan's stream while the lists (Algorithm 1) are built on
    // the auxiliary stream: neither needs the other's results, and the small
    // levels of the one leave room on the GPU for the other
    const bool fp32 = precision == SFMM_FP32;          // expansions and translations in FP32
    const bool dfe = precision == SFMM_MIXED || precision == SFMM_MIXED_DF;   // ... in double-float
    const bool near32 = precision == SFMM_FP32 || precision == SFMM_MIXED;    // FP32 near field
    const bool offsets = fp32 || dfe;                  // FP32 (hi, lo) offsets feed the near field
    const int ek = fp32 ? EXP_F32 : dfe ? EXP_DF : EXP_F64;
    const size_t esz = fp32 ? 4 : 8;                   // expansion storage: float, double or double-float
    if ((e = ensure(P->mpole, (size_t)nn * EXP_STRIDE * esz)) || (e = ensure(P->local, (size_t)nn * EXP_STRIDE * esz)))
        return cuda_fail(P, e, "alloc expansions");
    if ((e = cudaMemsetAsync(P->mpole.p, 0, (size_t)nn * EXP_STRIDE * esz, s))) return cuda_fail(P, e, "memset");
    if ((e = ensure(P->m2m_geo, (size_t)nn * xgeo_bytes(ek))) || (e = ensure(P->l2l_geo, (size_t)nn * xgeo_bytes(ek))))
        return cuda_fail(P, e, "alloc");
    if (fp32) {
        if ((e = ensure(P->geom32, (size_t)nn * 32))) return cuda_fail(P, e, "alloc");
        if ((e = launch_geom32((int)nn, P->n_geom.as<double>(), P->geom32.as<float>(), s)))
            return cuda_fail(P, e, "geometry32");
    }
    if (dfe) {
        // double-float frames per node, then the M2M / L2L parameters in double-float
        if ((e = ensure(P->framedf, (size_t)nn * frame_df_bytes()))) return cuda_fail(P, e, "alloc");
        if ((e = launch_frame_df((int)nn, T.d_nn, P->n_geom.as<double>(), P->framedf.p, s)) ||
            (e = launch_child_geo_df(T, P->framedf.p, P->logtab.as<float4>(), P->m2m_geo.p, P->l2l_geo.p, s)))
            return cuda_fail(P, e, "child geometry");
    } else if ((e = launch_child_geo(T, P->geom32.as<float>(), P->m2m_geo.p, P->l2l_geo.p, ek, s))) {
        return cuda_fail(P, e, "child geometry");
    }
    if ((e = cudaEventRecord(P->ev_fork, s)) || (e = cudaStreamWaitEvent(P->aux, P->ev_fork, 0)))
        return cuda_fail(P, e, "fork lists");
    if (offsets) {
        if ((e = ensure(P->soff, (size_t)N * 32))) return cuda_fail(P, e, "alloc");
        if ((e = launch_src_offsets(T, P->leaves_src.as<int>(), P->n_leaves, d_nls, P->src4.as<double4_32a>(),
                                    P->soff.as<float4>(), s)))
            return cuda_fail(P, e, "offsets");
    }
    if (adj && !adj_df) e = launch_p2m_adj(T, P->leaves_src.as<int>(), P->n_leaves, P->src4.as<double4_32a>(),
                                           P->dip4.as<double4_32a>(), P->mpole.as<double>(), p, s);
    else if (dfe) e = launch_p2m_df_leaf(T, P->leaves_src.as<int>(), P->n_leaves, d_nls, P->soff.as<float4>(),
                                         adj_df ? P->dip4.as<float4>() : nullptr, P->logtab.as<float4>(), p,
                                         P->mpole.p, s);
    else e = launch_p2m(T, P->leaves_src.as<int>(), P->n_leaves, d_nls, P->src4.as<double4_32a>(),
                        P->soff.as<float4>(), P->logtab.as<float4>(), P->mpole.p, p, ek, s);
    if (e) return cuda_fail(P, e, "P2M");
    // graph mode: every level up to the capacity, each launch sized by the level-width capacity
    const int depth = P->gm ? (int)P->cap.levels : (int)P->level_start.size() - 2;
    const int W = (int)P->cap.width;
    for (int l = depth - 1; l >= 0; --l) {
        if (dfe) e = P->gm ? launch_m2m_df(T, 0, W, l, p, P->m2m_geo.p, P->mpole.p, s)
                           : launch_m2m_df(T, P->level_start[l + 1], P->level_start[l + 2], l, p, P->m2m_geo.p,
                                           P->mpole.p, s);
        else e = P->gm ? launch_m2m(T, 0, W, l, p, P->tables.as<double>(), P->m2m_geo.p, P->mpole.p, ek, s)
                       : launch_m2m(T, P->level_start[l], P->level_start[l + 1], l, p, P->tables.as<double>(),
                                    P->m2m_geo.p, P->mpole.p, ek, s);
        if (e) return cuda_fail(P, e, "M2M");
    }
    tm.mark();
    // ---- lists on the auxiliary stream (its host synchronisation waits for the
    // walk only), joined back before M2L; the "lists" phase is the part of the walk
    // the up-pass did not hide
    if ((e = build_lists(P, T, P->opt.c_s, P->opt.c_t, P->aux))) {
        cudaStreamSynchronize(s);
        return cuda_fail(P, e, "lists");
    }
    // the evaluation's target and near-leaf offsets follow the P2P list on the auxiliary
    // stream (joined before the evaluation); M2L starts once its own list is sorted
    const uint32_t* p2p_s = P->p2p_alt ? P->p2p_s2.as<uint32_t>() : P->p2p_s.as<uint32_t>();
    if (offsets) {
        const uint64_t* p2p_t = P->p2p_alt ? P->p2p_t2.as<uint64_t>() : P->p2p_t.as<uint64_t>();
        if ((e = ensure(P->toff, (size_t)M * 32)) || (e = ensure(P->dc, (size_t)std::max<int64_t>(P->n_p2p, 1) * 32)))
            return cuda_fail(P, e, "alloc");
        if ((e = launch_eval32_prep(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->tgt4.as<double4_32a>(),
                                    P->toff.as<float4>(), p2p_t, p2p_s, P->n_p2p, P->d_p2p, P->dc.as<float4>(),
                                    P->aux)))
            return cuda_fail(P, e, "offsets");
    }
    // 1e-6 and 1e-10 paths: the near field needs none of the far field (their double-float
    // finish does), so it runs here, on the auxiliary stream, beside M2L and L2L
    unsigned long long* leaf_ctr = reinterpret_cast<unsigned long long*>(P->small.as<int64_t>() + 40);
    const bool near_early = near32 && !fp32 && !adj;
    const bool near_early_df = dfe && !near32 && !adj;
    if (near_early_df) {
        if ((e = ensure(P->nfbuf, (size_t)M * 48)) || (e = ensure(P->tleaf, (size_t)M * 4)))
            return cuda_fail(P, e, "alloc");
        if (P->timing) cudaEventRecord(P->ev_near[0], P->aux);
        if ((e = launch_eval_df(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->soff.as<float4>(),
                                P->toff.as<float4>(), P->dc.as<float4>(), P->tgt4.as<double4_32a>(), tperm,
                                P->p2p_off.as<int64_t>(), p2p_s, P->local.p, P->mpole.p, P->logtab.as<float4>(), p,
                                P->opt.zero_mean, psi, alpha, nullptr, nullptr, 0, nullptr, P->nfbuf.as<float4>(),
                                P->tleaf.as<int>(), P->framedf.p, M, EVAL_NEAR, leaf_ctr, P->aux)))
            return cuda_fail(P, e, "near field");
        if (P->timing) cudaEventRecord(P->ev_near[1], P->aux);
    }
    if (near_early) {
        if ((e = ensure(P->nfbuf, (size_t)M * 32)) || (e = ensure(P->tleaf, (size_t)M * 4)))
            return cuda_fail(P, e, "alloc");
        if (P->timing) cudaEventRecord(P->ev_near[0], P->aux);
        if ((e = launch_eval32(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->soff.as<float4>(),
                               P->toff.as<float4>(), P->dc.as<float4>(), P->tgt4.as<double4_32a>(), tperm,
                               P->p2p_off.as<int64_t>(), p2p_s, P->local.p, P->mpole.p, true, p, P->opt.zero_mean,
                               psi, alpha, src == tgt, P->nfbuf.as<float4>(), P->tleaf.as<int>(), P->framedf.p, M,
                               EVAL_NEAR, leaf_ctr, P->aux)))
            return cuda_fail(P, e, "near field");
        if (P->timing) cudaEventRecord(P->ev_near[1], P->aux);
    }
    if ((e = cudaEventRecord(P->ev_join, P->aux)) || (e = cudaStreamWaitEvent(s, P->ev_m2l, 0)))
        return cuda_fail(P, e, "join lists");
    tm.mark();
    // ---- M2L
    const uint32_t* m2l_s = P->m2l_alt ? P->m2l_s2.as<uint32_t>() : P->m2l_s.as<uint32_t>();
    const uint64_t* m2l_t = P->m2l_alt ? P->m2l_t2.as<uint64_t>() : P->m2l_t.as<uint64_t>();
    if ((e = ensure(P->m2l_geo, (size_t)std::max<int64_t>(P->n_m2l, 1) * xgeo_bytes(ek)))) return cuda_fail(P, e, "alloc");
    int* status = reinterpret_cast<int*>(P->small.as<int64_t>() + 20);
    if (dfe) {
        // double-float M2L, one thread per pair, summed per target box in FP64
        // accumulators; pairs with centres near antipodes go to the warp kernel
        const size_t nacc = (size_t)nn * EXP_STRIDE;
        uint32_t* n_left = reinterpret_cast<uint32_t*>(P->small.as<int64_t>() + 21);
        if ((e = ensure(P->m2l_acc, nacc * 8)) || (e = ensure(P->leftover, (size_t)std::max<int64_t>(P->n_m2l, 1) * 4)))
            return cuda_fail(P, e, "alloc");
        if ((e = cudaMemsetAsync(P->m2l_acc.p, 0, nacc * 8, s)) || (e = cudaMemsetAsync(n_left, 0, 4, s)))
            return cuda_fail(P, e, "memset");
        if ((e = launch_pair_geo_rho(T, P->framedf.p, P->logtab.as<float4>(), m2l_t, m2l_s, P->n_m2l, P->d_m2l,
                                     P->m2l_geo.p, s)))
            return cuda_fail(P, e, "pair geometry");
        if ((e = launch_m2l_pair(P->n_m2l, P->d_m2l, m2l_t, m2l_s, P->m2l_geo.p, P->mpole.p, p, P->m2l_acc.as<double>(),
                                 P->leftover.as<uint32_t>(), n_left, s)))
            return cuda_fail(P, e, "M2L");
        if ((e = launch_m2l_left_df(T, m2l_t, m2l_s, P->leftover.as<uint32_t>(), n_left, P->n_m2l, p,
                                    P->tables.as<double>(), P->mpole.p, P->m2l_acc.as<double>(), s)))
            return cuda_fail(P, e, "M2L (pairs near antipodes)");
    } else if ((e = cudaMemsetAsync(P->local.p, 0, (size_t)nn * EXP_STRIDE * esz, s)) ||
               (e = launch_pair_geo(T, P->geom32.as<float>(), m2l_t, m2l_s, P->n_m2l, P->d_m2l, P->m2l_geo.p, ek,
                                    s))) {
        return cuda_fail(P, e, "pair geometry");
    } else if (fp32 && P->opt.m2l_tensor_cores) {
        // tensor-core M2L; pairs it cannot take (centres near antipodes) go to a list for the warp kernel
        uint32_t* n_left = reinterpret_cast<uint32_t*>(P->small.as<int64_t>() + 21);
        uint32_t* tile_ctr = n_left + 1;              // zeroed by the same memset
        if ((e = ensure(P->leftover, (size_t)std::max<int64_t>(P->n_m2l, 1) * 4))) return cuda_fail(P, e, "alloc");
        if ((e = cudaMemsetAsync(P->small.as<int64_t>() + 20, 0, 16, s))) return cuda_fail(P, e, "memset");
        if ((e = launch_m2l_tc(P->n_m2l, m2l_t, m2l_s, P->m2l_geo.p, P->mpole.p, P->local.p, p, P->leftover.as<uint32_t>(),
                               n_left, tile_ctr, status, P->opt.wait_limit, s)))
            return cuda_fail(P, e, "M2L (tensor cores)");
        if ((e = launch_m2l_list(m2l_t, m2l_s, P->leftover.as<uint32_t>(), n_left, P->n_m2l, p, P->tables.as<double>(),
                                 P->m2l_geo.p, P->mpole.p, P->local.p, s)))
            return cuda_fail(P, e, "M2L (leftover pairs)");
    } else if ((e = launch_m2l(T, P->m2l_off.as<int64_t>(), m2l_s, p, P->tables.as<double>(), P->m2l_geo.p, P->mpole.p,
                               P->local.p, ek, s))) {
        return cuda_fail(P, e, "M2L");
    }
    tm.mark();
    // ---- L2L (double-float: each node's local is its M2L sum plus its parent's local translated)
    if (dfe) {
        for (int l = 0; l <= depth; ++l)
            if ((e = P->gm ? launch_l2l_df(T, 0, W, l, p, P->l2l_geo.p, P->m2l_acc.as<double>(), P->local.p, s)
                           : launch_l2l_df(T, P->level_start[l], P->level_start[l + 1], l, p, P->l2l_geo.p,
                                           P->m2l_acc.as<double>(), P->local.p, s)))
                return cuda_fail(P, e, "L2L");
    } else {
        for (int l = 1; l <= depth; ++l)
            if ((e = P->gm ? launch_l2l(T, 0, W, l, p, P->tables.as<double>(), P->l2l_geo.p, P->local.p, ek, s)
                           : launch_l2l(T, P->level_start[l], P->level_start[l + 1], l, p, P->tables.as<double>(),
                                        P->l2l_geo.p, P->local.p, ek, s)))
                return cuda_fail(P, e, "L2L");
    }
    tm.mark();
    // ---- evaluation (after the P2P list and the offsets of the auxiliary stream)
    if ((e = cudaStreamWaitEvent(s, P->ev_join, 0))) return cuda_fail(P, e, "join offsets");
    if (adj_df) e = launch_eval_df(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->soff.as<float4>(),
                                   P->toff.as<float4>(), P->dc.as<float4>(), P->tgt4.as<double4_32a>(), tperm,
                                   P->p2p_off.as<int64_t>(), p2p_s, P->local.p, P->mpole.p, P->logtab.as<float4>(), p,
                                   P->opt.zero_mean, psi, nullptr, P->dip4.as<float4>(), adj->w, adj->w_f32,
                                   adj->grad3, nullptr, nullptr, nullptr, M, EVAL_NEAR | EVAL_FINISH, leaf_ctr, s);
    else if (adj) e = launch_eval_adj(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, P->src4.as<double4_32a>(),
                                 P->dip4.as<double4_32a>(), P->tgt4.as<double4_32a>(), tperm, P->p2p_off.as<int64_t>(),
                                 p2p_s, P->local.as<double>(), P->mpole.as<double>(), p, P->opt.zero_mean, adj->w,
                                 adj->w_f32, psi, adj->grad3, leaf_ctr, s);
    else if (near32) {
        // 1e-6 path: the double-float finish on the near field's sums (the near field ran on the
        // auxiliary stream); all-FP32 path: the near field with its FP32 finish
        e = launch_eval32(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->soff.as<float4>(),
                          P->toff.as<float4>(), P->dc.as<float4>(), P->tgt4.as<double4_32a>(), tperm,
                          P->p2p_off.as<int64_t>(), p2p_s, P->local.p, P->mpole.p, !fp32, p, P->opt.zero_mean, psi,
                          alpha, src == tgt, P->nfbuf.as<float4>(), P->tleaf.as<int>(), P->framedf.p, M,
                          near_early ? EVAL_FINISH : EVAL_NEAR | EVAL_FINISH, leaf_ctr, s);
    }
    else if (dfe) e = launch_eval_df(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->soff.as<float4>(),
                                     P->toff.as<float4>(), P->dc.as<float4>(), P->tgt4.as<double4_32a>(), tperm,
                                     P->p2p_off.as<int64_t>(), p2p_s, P->local.p, P->mpole.p,
                                     P->logtab.as<float4>(), p, P->opt.zero_mean, psi, alpha, nullptr, nullptr, 0,
                                     nullptr, P->nfbuf.as<float4>(), P->tleaf.as<int>(), P->framedf.p, M,
                                     near_early_df ? EVAL_FINISH : EVAL_NEAR | EVAL_FINISH, leaf_ctr, s);
    else e = launch_eval(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, d_nlt, P->src4.as<double4_32a>(),
                         P->tgt4.as<double4_32a>(), tperm, P->p2p_off.as<int64_t>(), p2p_s, P->local.as<double>(),
                         P->mpole.as<double>(), p, P->opt.zero_mean, P->opt.sigma, psi, alpha, gamma, mu, leaf_ctr, s);
    if (e) return cuda_fail(P, e, "evaluation");
    if (P->gm) {          // no synchronisation: the caller reads the overflow flag after the work
        P->stats.launches = launch_total() - launches0;
        return SFMM_OK;
    }
    tm.mark();
    if (P->timing >= 2) {
        // near-field source-target pairs (for the throughput of the evaluation kernel)
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(P->small.as<int64_t>() + 16);
        if ((e = cudaMemsetAsync(cnt, 0, 8, s))) return cuda_fail(P, e, "memset");
        if ((e = launch_count_pairs(T, P->leaves_tgt.as<int>(), P->n_leaves_tgt, P->p2p_off.as<int64_t>(), p2p_s,
                                    cnt, s)))
            return cuda_fail(P, e, "count pairs");
        unsigned long long h = 0;
        if ((e = cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, s))) return cuda_fail(P, e, "copy");
        if ((e = cudaStreamSynchronize(s))) return cuda_fail(P, e, "sync");
        P->stats.p2p_interactions = (int64_t)h;
    }
    // the tensor-core M2L's status word comes back with the solve's one synchronisation
    const bool tc_status = fp32 && P->opt.m2l_tensor_cores;
    if (tc_status && (e = cudaMemcpyAsync(P->h_status, status, 4, cudaMemcpyDeviceToHost, s)))
        return cuda_fail(P, e, "status");
    if ((e = cudaStreamSynchronize(s))) return cuda_fail(P, e, "solve");
    if (tc_status && *P->h_status)
        return fail(P, SFMM_ETIMEOUT, "a bounded wait of the tensor-core M2L kernel ran out");
    tm.finish();
    if (P->timing && (near_early || near_early_df)) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P->ev_near[0], P->ev_near[1]) == cudaSuccess) P->stats.near_ms = ms;
    }
    P->stats.n_nodes = nn;
    P->stats.n_leaves = P->n_leaves;
    P->stats.depth = depth;
    P->stats.n_m2l = P->n_m2l;
    P->stats.n_p2p = P->n_p2p;
    P->stats.launches = launch_total() - launches0;
    return SFMM_OK;
}

sfmm_status check_args(sfmm_plan_s* P, const double* src, const void* q, int64_t N, const double* tgt, int64_t M)
{
    if (!P) return SFMM_EINVAL;
    if (N < 0 || M < 0) return fail(P, SFMM_EINVAL, "N and M must be non-negative");
    if (N > 0x7fffffffLL || M > 0x7fffffffLL) return fail(P, SFMM_EINVAL, "N and M must be below 2^31");
    if (N > 0 && (!src || !q)) return fail(P, SFMM_EINVAL, "src_xyz and q must be non-NULL when N > 0");
    if (M > 0 && !tgt) return fail(P, SFMM_EINVAL, "tgt_xyz must be non-NULL when M > 0");
    return SFMM_OK;
}

}  // namespace

// the solve for the other translation units (graph.cu)
sfmm_status solve_entry(sfmm_plan_s* P, const double* src, const void* q, int64_t N, const double* tgt, int64_t M,
                        double* psi, double* alpha)
{
    return solve(P, src, q, N, tgt, M, psi, alpha);
}

sfmm_status plan_error(sfmm_plan_s* P, sfmm_status st, const std::string& msg) { return fail(P, st, msg); }

void set_process_error(const std::string& msg)
{
    std::lock_guard<std::mutex> g(g_err_mu);
    g_plan_err = msg;
}
}  // namespace sfmm

using namespace sfmm;

extern "C" {

sfmm_status sfmm_default_options(sfmm_options* opt)
{
    if (!opt) return SFMM_EINVAL;
    memset(opt, 0, sizeof *opt);
    opt->leaf_size = 32;
    opt->c_s = 2.0;
    opt->c_t = 0.5;
    opt->precision = SFMM_FP64;
    opt->m2l_tensor_cores = 1;
    return SFMM_OK;
}

sfmm_status sfmm_plan(sfmm_plan_t* out, int max_depth, int order_p, double tol, const sfmm_options* opt)
{
    auto plan_fail = [](const char* m) {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_plan_err = m;
        return SFMM_EINVAL;
    };
    if (!out) return plan_fail("out is NULL");
    *out = nullptr;
    if (max_depth < 0 || max_depth > ORDER_MAX) return plan_fail("max_depth must be in 0..29");
    if (order_p < 0 || order_p > PMAX) return plan_fail("order_p must be in 0..32");
    if (order_p == 0 && !(tol > 0.0 && tol < 1.0)) return plan_fail("tol must be in (0, 1) when order_p == 0");
    sfmm_options o;
    sfmm_default_options(&o);
    if (opt) {
        o = *opt;
        if (o.leaf_size == 0) o.leaf_size = 32;
        if (o.c_s == 0.0) o.c_s = 2.0;
        if (o.c_t == 0.0) o.c_t = 0.5;
    }
    if (o.leaf_size < 1) return plan_fail("leaf_size must be >= 1");
    if (!(o.c_s > 1.0)) return plan_fail("c_s must be > 1 (Sec. 3.5)");
    if (!(o.c_t > 0.0 && o.c_t < 1.0)) return plan_fail("c_t must be in (0, 1) (Sec. 3.5)");
    if (o.precision != SFMM_FP64 && o.precision != SFMM_MIXED && o.precision != SFMM_MIXED_DF &&
        o.precision != SFMM_FP32)
        return plan_fail("unknown precision");
    if (o.n_max < 0 || o.m_max < 0) return plan_fail("n_max and m_max must be >= 0");
    if (!(o.sigma >= 0.0 && o.sigma < 1.5707963267948966)) return plan_fail("sigma must be in [0, pi/2)");
    if (o.wait_limit < 0) return plan_fail("wait_limit must be >= 0");
    if (o.sigma > 0.0 && o.precision != SFMM_FP64)
        return plan_fail("sigma > 0 (Near Particle Model) runs on the FP64 path only (precision SFMM_FP64)");
    auto* P = new (std::nothrow) sfmm_plan_s();
    if (!P) return SFMM_ENOMEM;
    P->max_depth = max_depth;
    P->p = order_p ? order_p : p_from_tol(tol);
    P->tol = tol;
    P->opt = o;
    P->stream = static_cast<cudaStream_t>(o.stream);
    std::vector<double> h(2 * PMAX * PMAX);
    fill_tables(h.data());
    float lt[129 * 4];
    fill_log_table(lt);
    cudaError_t e;
    if ((e = cudaMallocHost(&P->h_status, sizeof(int))) || (e = cudaStreamCreateWithFlags(&P->aux, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&P->ev_m2l, cudaEventDisableTiming)) ||
        (e = cudaEventCreate(&P->ev_near[0])) || (e = cudaEventCreate(&P->ev_near[1]))) {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_plan_err = std::string("CUDA error at plan time: ") + cudaGetErrorString(e);
        sfmm_destroy(P);
        return SFMM_ECUDA;
    }
    if ((e = ensure(P->tables, h.size() * 8)) ||
        (e = cudaMemcpy(P->tables.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice)) ||
        (e = ensure(P->logtab, sizeof lt)) || (e = cudaMemcpy(P->logtab.p, lt, sizeof lt, cudaMemcpyHostToDevice))) {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_plan_err = std::string("CUDA error at plan time: ") + cudaGetErrorString(e);
        delete P;
        return e == cudaErrorMemoryAllocation ? SFMM_ENOMEM : SFMM_ECUDA;
    }
    if (o.n_max > 0 || o.m_max > 0) {
        const int64_t N = o.n_max, M = o.m_max;
        if ((e = ensure(P->skeys, N * 8)) || (e = ensure(P->skeys2, N * 8)) || (e = ensure(P->sperm, N * 4)) ||
            (e = ensure(P->sperm2, N * 4)) || (e = ensure(P->src4, N * 32)) || (e = ensure(P->tkeys, M * 8)) ||
            (e = ensure(P->tkeys2, M * 8)) || (e = ensure(P->tperm, M * 4)) || (e = ensure(P->tperm2, M * 4)) ||
            (e = ensure(P->tgt4, M * 32)) || (e = ensure(P->tmp, radix_tmp_bytes(std::max(N, M)))) ||
            (e = ensure(P->ttmp, radix_tmp_bytes(M)))) {
            std::lock_guard<std::mutex> g(g_err_mu);
            g_plan_err = std::string("workspace allocation failed: ") + cudaGetErrorString(e);
            sfmm_destroy(P);
            return SFMM_ENOMEM;
        }
    }
    *out = P;
    return SFMM_OK;
}

sfmm_status sfmm_potential(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N, const double* tgt_xyz,
                           int64_t M, double* psi)
{
    sfmm_status st = check_args(plan, src_xyz, q, N, tgt_xyz, M);
    if (st != SFMM_OK) return st;
    if (M > 0 && !psi) return fail(plan, SFMM_EINVAL, "psi must be non-NULL");
    return solve(plan, src_xyz, q, N, tgt_xyz, M, psi, nullptr);
}

sfmm_status sfmm_deflection(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N, const double* tgt_xyz,
                            int64_t M, double* psi, double* alpha)
{
    sfmm_status st = check_args(plan, src_xyz, q, N, tgt_xyz, M);
    if (st != SFMM_OK) return st;
    if (M > 0 && !alpha) return fail(plan, SFMM_EINVAL, "alpha must be non-NULL");
    return solve(plan, src_xyz, q, N, tgt_xyz, M, psi, alpha);
}

sfmm_status sfmm_deflection_batch(sfmm_plan_t plan, int n_shells, const double* const* src_xyz,
                                  const void* const* q, const int64_t* N, const double* const* tgt_xyz,
                                  const int64_t* M, double* const* psi, double* const* alpha, int lanes)
{
    if (!plan) return SFMM_EINVAL;
    if (n_shells < 0) return fail(plan, SFMM_EINVAL, "n_shells must be >= 0");
    if (n_shells == 0) return SFMM_OK;
    if (!src_xyz || !q || !N || !tgt_xyz || !M || !alpha) return fail(plan, SFMM_EINVAL, "NULL array of shells");
    for (int i = 0; i < n_shells; ++i) {
        sfmm_status st = check_args(plan, src_xyz[i], q[i], N[i], tgt_xyz[i], M[i]);
        if (st != SFMM_OK) return st;
        if (M[i] > 0 && !alpha[i]) return fail(plan, SFMM_EINVAL, "alpha must be non-NULL for every shell with M > 0");
    }
    lanes = std::max(1, std::min(std::min(lanes, 8), n_shells));
    cudaError_t e;
    // lane solvers: the plan's settings, each on its own non-blocking stream
    while ((int)plan->lanes.size() < lanes) {
        sfmm_options o = plan->opt;
        cudaStream_t st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) return cuda_fail(plan, e, "lane stream");
        o.stream = st;
        o.n_max = o.m_max = 0;
        sfmm_plan_t L = nullptr;
        sfmm_status ps = sfmm_plan(&L, plan->max_depth, plan->p, plan->tol, &o);
        if (ps != SFMM_OK) {
            cudaStreamDestroy(st);
            return fail(plan, ps, "could not create a batch lane");
        }
        L->owns_stream = true;
        plan->lanes.push_back(L);
    }
    // the lanes start after the work already queued on the plan's stream
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) || (e = cudaEventRecord(ev, plan->stream)))
        return cuda_fail(plan, e, "batch event");
    for (int l = 0; l < lanes; ++l)
        if ((e = cudaStreamWaitEvent(plan->lanes[l]->stream, ev, 0))) {
            cudaEventDestroy(ev);
            return cuda_fail(plan, e, "batch wait");
        }
    // largest shells first; each lane's host thread takes the next shell
    std::vector<int> order(n_shells);
    for (int i = 0; i < n_shells; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return N[a] + M[a] > N[b] + M[b]; });
    std::atomic<int> next{0};
    std::mutex mu;
    sfmm_status first = SFMM_OK;
    std::string msg;
    int dev = 0;
    cudaGetDevice(&dev);
    auto work = [&](sfmm_plan_s* L) {
        cudaSetDevice(dev);
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= n_shells) return;
            const int i = order[k];
            const sfmm_status st = solve(L, src_xyz[i], q[i], N[i], tgt_xyz[i], M[i], psi ? psi[i] : nullptr, alpha[i]);
            if (st != SFMM_OK) {
                std::lock_guard<std::mutex> g(mu);
                if (first == SFMM_OK) { first = st; msg = "shell " + std::to_string(i) + ": " + L->err; }
                next.store(n_shells);
                return;
            }
        }
    };
    std::vector<std::thread> th;
    for (int l = 1; l < lanes; ++l) th.emplace_back(work, plan->lanes[l]);
    work(plan->lanes[0]);
    for (auto& t : th) t.join();
    // and the plan's stream continues after all of them
    for (int l = 0; l < lanes; ++l) {
        if ((e = cudaEventRecord(ev, plan->lanes[l]->stream)) || (e = cudaStreamWaitEvent(plan->stream, ev, 0))) break;
    }
    cudaEventDestroy(ev);
    if (first != SFMM_OK) return fail(plan, first, msg.c_str());
    if (e) return cuda_fail(plan, e, "batch join");
    return SFMM_OK;
}

sfmm_status sfmm_shear(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N, const double* tgt_xyz,
                       int64_t M, double* psi, double* alpha, double* gamma, double* mu)
{
    sfmm_status st = check_args(plan, src_xyz, q, N, tgt_xyz, M);
    if (st != SFMM_OK) return st;
    if (M > 0 && !gamma) return fail(plan, SFMM_EINVAL, "gamma must be non-NULL");
    if (plan->opt.sigma > 0.0) return fail(plan, SFMM_EINVAL, "sfmm_shear supports point masses only (sigma == 0)");
    return solve(plan, src_xyz, q, N, tgt_xyz, M, psi, alpha, nullptr, gamma, mu);
}

sfmm_status sfmm_adjoint(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N, const double* tgt_xyz,
                         int64_t M, const double* g_psi, const double* g_alpha, double* grad_q, double* grad_src)
{
    sfmm_status st = check_args(plan, src_xyz, q, N, tgt_xyz, M);
    if (st != SFMM_OK) return st;
    if (N > 0 && !grad_q && !grad_src) return fail(plan, SFMM_EINVAL, "grad_q or grad_src must be non-NULL");
    if (plan->opt.sigma > 0.0) return fail(plan, SFMM_EINVAL, "sfmm_adjoint supports point masses only (sigma == 0)");
    if (N == 0) return SFMM_OK;
    cudaStream_t s = plan->stream;
    cudaError_t e;
    if (M == 0 || (!g_psi && !g_alpha)) {           // no loss terms: zero gradients
        if (grad_q && (e = cudaMemsetAsync(grad_q, 0, (size_t)N * 8, s))) return cuda_fail(plan, e, "memset");
        if (grad_src && (e = cudaMemsetAsync(grad_src, 0, (size_t)N * 24, s))) return cuda_fail(plan, e, "memset");
        if ((e = cudaStreamSynchronize(s))) return cuda_fail(plan, e, "sync");
        return SFMM_OK;
    }
    if ((e = ensure(plan->adj_h, (size_t)M * 8)) || (e = ensure(plan->adj_g, (size_t)M * 24)))
        return cuda_fail(plan, e, "alloc adjoint sources");
    k_adjoint_prep<<<grid_for(M), 256, 0, s>>>(tgt_xyz, M, g_psi, g_alpha, plan->adj_h.as<double>(),
                                               plan->adj_g.as<double>());
    count_launch();
    if ((e = cudaGetLastError())) return cuda_fail(plan, e, "adjoint sources");
    // the forward targets carry the charges and dipoles; the field is evaluated at the forward sources
    AdjIO adj{plan->adj_g.as<double>(), q, plan->opt.q_f32, grad_src};
    return solve(plan, tgt_xyz, plan->adj_h.p, M, src_xyz, N, grad_q, nullptr, &adj);
}

sfmm_status sfmm_deflection_host(sfmm_plan_t plan, const double* src_xyz, const void* q, int64_t N,
                                 const double* tgt_xyz, int64_t M, double* psi, double* alpha)
{
    sfmm_status st = check_args(plan, src_xyz, q, N, tgt_xyz, M);
    if (st != SFMM_OK) return st;
    if (M > 0 && !alpha) return fail(plan, SFMM_EINVAL, "alpha must be non-NULL");
    sfmm_plan_s* P = plan;
    cudaStream_t s = P->stream;
    cudaError_t e;
    const size_t qb = P->opt.q_f32 ? 4 : 8;
    if ((e = ensure(P->h_src, std::max<int64_t>(N, 1) * 24)) || (e = ensure(P->h_q, std::max<int64_t>(N, 1) * qb)) ||
        (e = ensure(P->h_tgt, std::max<int64_t>(M, 1) * 24)) || (e = ensure(P->h_alpha, std::max<int64_t>(M, 1) * 16)) ||
        (psi && (e = ensure(P->h_psi, std::max<int64_t>(M, 1) * 8))))
        return cuda_fail(P, e, "alloc staging");
    // The targets are copied on the auxiliary stream, where the solve handles them
    // (forked here, after earlier work on the plan's stream), so that copy overlaps
    // the source copies and the sources' keys and sort.
    if ((e = cudaEventRecord(P->ev_fork, s)) || (e = cudaStreamWaitEvent(P->aux, P->ev_fork, 0)))
        return cuda_fail(P, e, "fork");
    if (M > 0 && (e = cudaMemcpyAsync(P->h_tgt.p, tgt_xyz, M * 24, cudaMemcpyHostToDevice, P->aux)))
        return cuda_fail(P, e, "copy targets");
    if (N > 0 && ((e = cudaMemcpyAsync(P->h_src.p, src_xyz, N * 24, cudaMemcpyHostToDevice, s)) ||
                  (e = cudaMemcpyAsync(P->h_q.p, q, N * qb, cudaMemcpyHostToDevice, s)))) {
        cudaStreamSynchronize(P->aux);
        return cuda_fail(P, e, "copy inputs");
    }
    P->forked = true;
    st = solve(P, P->h_src.as<double>(), P->h_q.p, N, P->h_tgt.as<double>(), M, psi ? P->h_psi.as<double>() : nullptr,
               P->h_alpha.as<double>());
    P->forked = false;
    // every path out of the solve leaves no copy of the caller's targets in flight
    if ((e = cudaStreamSynchronize(P->aux)) && st == SFMM_OK) return cuda_fail(P, e, "sync");
    if (st != SFMM_OK) return st;
    if (M > 0) {
        if ((e = cudaMemcpyAsync(alpha, P->h_alpha.p, M * 16, cudaMemcpyDeviceToHost, s)))
            return cuda_fail(P, e, "copy alpha");
        if (psi && (e = cudaMemcpyAsync(psi, P->h_psi.p, M * 8, cudaMemcpyDeviceToHost, s)))
            return cuda_fail(P, e, "copy psi");
        if ((e = cudaStreamSynchronize(s))) return cuda_fail(P, e, "sync");
    }
    return SFMM_OK;
}

void sfmm_destroy(sfmm_plan_t plan)
{
    if (!plan) return;
    Buf* all[] = {&plan->skeys, &plan->skeys2, &plan->sperm, &plan->sperm2, &plan->src4, &plan->tkeys, &plan->tkeys2,
                  &plan->tperm, &plan->tperm2, &plan->tgt4, &plan->h_src, &plan->h_q, &plan->h_tgt, &plan->h_psi,
                  &plan->h_alpha, &plan->tmp, &plan->flags, &plan->pos, &plan->small, &plan->n_prefix,
                  &plan->n_level, &plan->n_first, &plan->n_count, &plan->n_child0, &plan->n_parent, &plan->n_geom,
                  &plan->n_tfirst, &plan->n_tcount, &plan->mpole, &plan->local, &plan->tables, &plan->fa, &plan->fb,
                  &plan->act, &plan->c_next, &plan->c_m2l, &plan->c_p2p, &plan->o_next, &plan->o_m2l, &plan->o_p2p,
                  &plan->m2l_t, &plan->m2l_s, &plan->m2l_t2, &plan->m2l_s2, &plan->p2p_t, &plan->p2p_s,
                  &plan->p2p_t2, &plan->p2p_s2, &plan->m2l_off, &plan->p2p_off, &plan->leaves_src,
                  &plan->leaves_tgt, &plan->m2l_geo, &plan->m2m_geo, &plan->l2l_geo, &plan->soff,
                  &plan->toff, &plan->dc, &plan->leftover, &plan->geom32, &plan->macn, &plan->logtab,
                  &plan->ttmp, &plan->dip4, &plan->adj_h, &plan->adj_g, &plan->macn32, &plan->m2l_acc,
                  &plan->framedf, &plan->dcnt, &plan->nfbuf, &plan->tleaf};
    if (plan->aux) cudaStreamSynchronize(plan->aux);
    graph_release(plan);
    for (sfmm_plan_s* L : plan->lanes) sfmm_destroy(L);
    plan->lanes.clear();
    if (plan->owns_stream && plan->stream) {
        cudaStreamSynchronize(plan->stream);
        cudaStreamDestroy(plan->stream);
    }
    for (Buf* b : all) release(*b);
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    if (plan->ev_m2l) cudaEventDestroy(plan->ev_m2l);
    for (cudaEvent_t ev : plan->ev_near)
        if (ev) cudaEventDestroy(ev);
    if (plan->aux) cudaStreamDestroy(plan->aux);
    if (plan->h_status) cudaFreeHost(plan->h_status);
    delete plan;
}

const char* sfmm_last_error(sfmm_plan_t plan)
{
    if (!plan) {
        std::lock_guard<std::mutex> g(g_err_mu);
        return g_plan_err.c_str();
    }
    return plan->err.c_str();
}

int sfmm_order(sfmm_plan_t plan) { return plan ? plan->p : 0; }

sfmm_status sfmm_get_stats(sfmm_plan_t plan, sfmm_stats* out)
{
    if (!plan || !out) return SFMM_EINVAL;
    *out = plan->stats;
    return SFMM_OK;
}

sfmm_status sfmm_set_wait_limit(sfmm_plan_t plan, int polls)
{
    if (!plan) return SFMM_EINVAL;
    if (polls < 0) return fail(plan, SFMM_EINVAL, "wait limit must be >= 0");
    plan->opt.wait_limit = polls;
    return SFMM_OK;
}

sfmm_status sfmm_set_timing(sfmm_plan_t plan, int on)
{
    if (!plan) return SFMM_EINVAL;
    if (on < 0 || on > 2) return fail(plan, SFMM_EINVAL, "timing level must be 0, 1 or 2");
    plan->timing = on;
    return SFMM_OK;
}

sfmm_status sfmm_debug_copy(sfmm_plan_t plan, int which, void* dst, int64_t bytes, int64_t* bytes_needed)
{
    if (!plan) return SFMM_EINVAL;
    sfmm_plan_s* P = plan;
    const int64_t N = P->last_N, M = P->last_M, nn = P->n_nodes;
    const int p = P->p;
    const void* srcp = nullptr;
    int64_t need = 0;
    Buf tmpbuf;
    switch (which) {
    case SFMM_ARR_SRC_KEYS: srcp = P->skeys_alt ? P->skeys2.p : P->skeys.p; need = N * 8; break;
    case SFMM_ARR_SRC_PERM: srcp = P->skeys_alt ? P->sperm2.p : P->sperm.p; need = N * 4; break;
    case SFMM_ARR_TGT_KEYS: srcp = P->tkeys_alt ? P->tkeys2.p : P->tkeys.p; need = M * 8; break;
    case SFMM_ARR_NODE_PREFIX: srcp = P->n_prefix.p; need = nn * 8; break;
    case SFMM_ARR_NODE_LEVEL: srcp = P->n_level.p; need = nn * 4; break;
    case SFMM_ARR_NODE_CHILD0: srcp = P->n_child0.p; need = nn * 4; break;
    case SFMM_ARR_NODE_PARENT: srcp = P->n_parent.p; need = nn * 4; break;
    case SFMM_ARR_NODE_GEOM: need = nn * 11 * 8; break;
    case SFMM_ARR_NODE_RANGE: need = nn * 8; break;
    case SFMM_ARR_NODE_TRANGE: need = nn * 8; break;
    case SFMM_ARR_MULTIPOLE: case SFMM_ARR_LOCAL: need = nn * (2 * p + 2) * 8; break;
    case SFMM_ARR_M2L: need = P->n_m2l * 8; break;
    case SFMM_ARR_P2P: need = P->n_p2p * 8; break;
    case SFMM_ARR_SRC_OFFSETS:
        srcp = P->soff.p;
        need = P->opt.precision == SFMM_FP64 || !srcp ? 0 : N * 32;
        break;
    case SFMM_ARR_TGT_OFFSETS:
        srcp = P->toff.p;
        need = P->opt.precision == SFMM_FP64 || !srcp ? 0 : M * 32;
        break;
    default: return fail(P, SFMM_EINVAL, "unknown array");
    }
    if (bytes_needed) *bytes_needed = need;
    if (!dst) return SFMM_OK;
    if (bytes < need) return fail(P, SFMM_EINVAL, "destination too small");
    if (need == 0) return SFMM_OK;
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e) return cuda_fail(P, e, "sync");
    if (srcp) {
        e = cudaMemcpy(dst, srcp, need, cudaMemcpyDeviceToHost);
        return e ? cuda_fail(P, e, "copy") : SFMM_OK;
    }
    std::vector<char> h;
    char* d = static_cast<char*>(dst);
    if (which == SFMM_ARR_NODE_GEOM) {
        std::vector<double> g((size_t)nn * GEOM_STRIDE);
        if ((e = cudaMemcpy(g.data(), P->n_geom.p, g.size() * 8, cudaMemcpyDeviceToHost))) return cuda_fail(P, e, "copy");
        double* o = reinterpret_cast<double*>(d);
        for (int64_t i = 0; i < nn; ++i)
            for (int k = 0; k < 11; ++k) o[i * 11 + k] = g[i * GEOM_STRIDE + k];
        return SFMM_OK;
    }
    if (which == SFMM_ARR_NODE_RANGE || which == SFMM_ARR_NODE_TRANGE) {
        std::vector<int> a(nn), b(nn);
        const Buf& fa = which == SFMM_ARR_NODE_RANGE ? P->n_first : P->n_tfirst;
        const Buf& fb = which == SFMM_ARR_NODE_RANGE ? P->n_count : P->n_tcount;
        if ((e = cudaMemcpy(a.data(), fa.p, nn * 4, cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(b.data(), fb.p, nn * 4, cudaMemcpyDeviceToHost)))
            return cuda_fail(P, e, "copy");
        int* o = reinterpret_cast<int*>(d);
        for (int64_t i = 0; i < nn; ++i) { o[2 * i] = a[i]; o[2 * i + 1] = b[i]; }
        return SFMM_OK;
    }
    if (which == SFMM_ARR_MULTIPOLE || which == SFMM_ARR_LOCAL) {
        if ((e = ensure(tmpbuf, need))) return cuda_fail(P, e, "alloc");
        const Buf& in = which == SFMM_ARR_MULTIPOLE ? P->mpole : P->local;
        if ((e = launch_unscale((int)nn, P->n_geom.as<double>(), in.p, tmpbuf.as<double>(), p,
                                which == SFMM_ARR_LOCAL,
                                P->opt.precision == SFMM_FP32 ? EXP_F32 : P->opt.precision == SFMM_FP64 ? EXP_F64 : EXP_DF,
                                P->stream)) ||
            (e = cudaStreamSynchronize(P->stream)) || (e = cudaMemcpy(dst, tmpbuf.p, need, cudaMemcpyDeviceToHost))) {
            release(tmpbuf);
            return cuda_fail(P, e, "unscale");
        }
        release(tmpbuf);
        return SFMM_OK;
    }
    // lists: (source, target) pairs grouped by target
    const int64_t np = which == SFMM_ARR_M2L ? P->n_m2l : P->n_p2p;
    const bool alt = which == SFMM_ARR_M2L ? P->m2l_alt : P->p2p_alt;
    const Buf& bt = which == SFMM_ARR_M2L ? (alt ? P->m2l_t2 : P->m2l_t) : (alt ? P->p2p_t2 : P->p2p_t);
    const Buf& bs = which == SFMM_ARR_M2L ? (alt ? P->m2l_s2 : P->m2l_s) : (alt ? P->p2p_s2 : P->p2p_s);
    std::vector<uint64_t> t(np);
    std::vector<uint32_t> sv(np);
    if ((e = cudaMemcpy(t.data(), bt.p, np * 8, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(sv.data(), bs.p, np * 4, cudaMemcpyDeviceToHost)))
        return cuda_fail(P, e, "copy");
    int* o = reinterpret_cast<int*>(d);
    for (int64_t i = 0; i < np; ++i) { o[2 * i] = (int)sv[i]; o[2 * i + 1] = (int)t[i]; }
    return SFMM_OK;
}

sfmm_status sfmm_keys(const double* xyz, int64_t n, uint64_t* keys, void* stream)
{
    if (n < 0 || (n > 0 && (!xyz || !keys))) return SFMM_EINVAL;
    cudaError_t e = launch_keys(xyz, n, keys, nullptr, static_cast<cudaStream_t>(stream));
    return e ? SFMM_ECUDA : SFMM_OK;
}

}  // extern "C"
