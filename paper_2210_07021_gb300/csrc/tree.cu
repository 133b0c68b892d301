// The adaptive 12-root quad-tree of Sec. 3.1 and its box geometry.
//
// Division rule (Sec. 3.1, steps 1-3): the 12 HEALPix base boxes hold the
// particles by key; a box holding more than m particles is divided into its 4
// children (always 4, empty or not) until no box holds more than m, or the
// level reaches the maximum depth (r_max = 29 by default).  Built level by level
// from the key-sorted particles: a child's particle range is found by binary
// search inside its parent's range.  Nodes are numbered by level, then by
// pixel index.
//
// Geometry (Sec. 3.1 frame K_P, Sec. 3.5 radius): a box's centre is its HEALPix
// pixel centre; its frame has zenith e_r(centre) and azimuth reference
// e_theta(centre); its radius R is the largest angle from the centre to the
// pixel's 4 corners (the corners realise the covering radius of a HEALPix
// pixel), plus 2e-15 rad for the rounding of the keys.  r = tan(R/2) is the
// scale of the stereographic variable z = tan(theta/2) e^{i phi} inside the box.
#include "common.cuh"

#include <algorithm>

namespace sfmm {

namespace {

__constant__ int c_jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
__constant__ int c_jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t lo, int64_t hi, uint64_t v)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t compact_bits(uint64_t v)
{
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
    v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
    v = (v | (v >> 16)) & 0x00000000FFFFFFFFull;
    return v;
}

// Point at continuous face coordinates (X, Y) in [0, nside]^2 of base pixel
// `face` (the inverse of the ang2pix mapping): unit vector, plus cos/sin of
// its polar angle and cos/sin of its azimuth.
__device__ void facexy2vec(int order, int face, double X, double Y, double v[3], double* ct, double* st,
                           double* cp, double* sp)
{
    const double nside = ldexp(1.0, order);
    const double jr = c_jrll[face] * nside - X - Y;
    double nr, z, s;
    if (jr < nside) {
        nr = jr;
        const double t = nr * nr / (3.0 * nside * nside);   // 1 - z
        z = 1.0 - t;
        s = sqrt(t * (2.0 - t));
    } else if (jr > 3.0 * nside) {
        nr = 4.0 * nside - jr;
        const double t = nr * nr / (3.0 * nside * nside);   // 1 + z
        z = t - 1.0;
        s = sqrt(t * (2.0 - t));
    } else {
        nr = nside;
        z = (2.0 * nside - jr) * 2.0 / (3.0 * nside);
        s = sqrt((1.0 - z) * (1.0 + z));
    }
    double c_, s_;
    if (nr > 0.0) sincospi(0.25 * (c_jpll[face] + (X - Y) / nr), &s_, &c_);
    else { s_ = 0.0; c_ = 1.0; }
    v[0] = s * c_; v[1] = s * s_; v[2] = z;
    *ct = z; *st = s; *cp = c_; *sp = s_;
}

__global__ void k_level0(const uint64_t* __restrict__ keys, int64_t n, uint64_t* prefix, int* level, int* first,
                         int* count, int* child0, int* parent)
{
    const int f = threadIdx.x;
    if (f >= 12) return;
    const uint64_t lo = (uint64_t)f << (2 * ORDER_MAX), hi = (uint64_t)(f + 1) << (2 * ORDER_MAX);
    const int64_t a = lower_bound_u64(keys, 0, n, lo);
    const int64_t b = lower_bound_u64(keys, a, n, hi);
    prefix[f] = (uint64_t)f;
    level[f] = 0;
    first[f] = (int)a;
    count[f] = (int)(b - a);
    child0[f] = -1;
    parent[f] = -1;
}

// Graph mode (dc != NULL): the level's bounds come from dc->level, the launch
// covers `width` (the level-width capacity) and the flags beyond the level are
// zero, so that a scan over the whole capacity is the scan of the level.
__global__ void k_split_flags(const int* __restrict__ count, int a, int b, int lvl, int m, int max_depth,
                              int64_t* __restrict__ flags, DevCounts* dc, int64_t width)
{
    if (dc) {
        a = (int)dc->level[lvl];
        b = (int)dc->level[lvl + 1];
        if (blockIdx.x == 0 && threadIdx.x == 0 && b - a > width) dc->overflow = 1;
    } else {
        width = b - a;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < width; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i < b - a && count[a + i] > m && lvl < max_depth) ? 1 : 0;
}

__global__ void k_counts_init(DevCounts* dc)
{
    if (threadIdx.x < 32) dc->level[threadIdx.x] = threadIdx.x == 0 ? 0 : 12;
    if (threadIdx.x == 0) { dc->nn = 12; dc->n_leaves = 0; dc->n_leaves_tgt = 0; dc->overflow = 0; }
}

// Graph mode: the next level's end from the scan of the split flags (its total),
// or an overflow if the nodes would not fit the capacity (`last`: the deepest
// level the capacity allows; a split there is an overflow too).
__global__ void k_level_end(DevCounts* dc, int lvl, const int64_t* __restrict__ total, int64_t node_cap, int last)
{
    const int64_t b = dc->level[lvl + 1];
    int64_t nb = b + 4 * *total;
    // after an overflow the tree stops growing: the nodes built so far stay a
    // consistent tree (unsplit nodes are leaves), so every later kernel stays in bounds
    if (dc->overflow || nb > node_cap || (last && *total > 0)) {
        dc->overflow = 1;
        nb = b;
    }
    dc->level[lvl + 2] = nb;
    dc->nn = nb;
}

__global__ void k_make_children(const uint64_t* __restrict__ keys, int a, int b, int lvl,
                                const int64_t* __restrict__ flags, const int64_t* __restrict__ pos,
                                uint64_t* prefix, int* level, int* first, int* count, int* child0, int* parent,
                                const DevCounts* dc)
{
    if (dc) {
        if (dc->overflow) return;
        a = (int)dc->level[lvl];
        b = (int)dc->level[lvl + 1];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b - a; i += (int64_t)gridDim.x * blockDim.x) {
        const int node = a + (int)i;
        if (!flags[i]) continue;
        const int c0 = b + 4 * (int)pos[i];
        child0[node] = c0;
        const int shift = 2 * (ORDER_MAX - (lvl + 1));
        const uint64_t pf = prefix[node] * 4ull;
        const int64_t lo = first[node], hi = lo + count[node];
        int64_t starts[5];
        starts[0] = lo;
        starts[4] = hi;
        for (int c = 1; c < 4; ++c) starts[c] = lower_bound_u64(keys, starts[c - 1], hi, (pf + c) << shift);
        for (int c = 0; c < 4; ++c) {
            prefix[c0 + c] = pf + c;
            level[c0 + c] = lvl + 1;
            first[c0 + c] = (int)starts[c];
            count[c0 + c] = (int)(starts[c + 1] - starts[c]);
            child0[c0 + c] = -1;
            parent[c0 + c] = node;
        }
    }
}

__global__ void k_geometry(int n_cap, const int64_t* d_nn, const uint64_t* __restrict__ prefix,
                           const int* __restrict__ level, double* __restrict__ geom)
{
    const int64_t n_nodes = dcount(d_nn, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const int order = level[i];
        const uint64_t pix = prefix[i];
        const int face = (int)(pix >> (2 * order));
        const uint64_t ipf = pix & ((1ull << (2 * order)) - 1ull);
        const double ix = (double)compact_bits(ipf), iy = (double)compact_bits(ipf >> 1);
        double c[3], ct, st, cp, sp;
        facexy2vec(order, face, ix + 0.5, iy + 0.5, c, &ct, &st, &cp, &sp);
        double chord2 = 0.0;
        for (int k = 0; k < 4; ++k) {
            double v[3], a, b, e, f;
            facexy2vec(order, face, ix + (k & 1), iy + (k >> 1), v, &a, &b, &e, &f);
            const double dx = v[0] - c[0], dy = v[1] - c[1], dz = v[2] - c[2];
            chord2 = fmax(chord2, dx * dx + dy * dy + dz * dz);
        }
        const double R = 2.0 * asin(fmin(1.0, 0.5 * sqrt(chord2))) + 2e-15;
        double* g = geom + (size_t)i * GEOM_STRIDE;
        g[0] = c[0]; g[1] = c[1]; g[2] = c[2];
        g[3] = ct * cp; g[4] = ct * sp; g[5] = -st;     // e_theta at the centre
        g[6] = -sp; g[7] = cp; g[8] = 0.0;              // e_phi at the centre
        g[9] = R;
        g[10] = tan(0.5 * R);
        g[11] = 0.0;
    }
}

__global__ void k_target_ranges(int n_cap, const int64_t* d_nn, const uint64_t* __restrict__ prefix,
                                const int* __restrict__ level, const uint64_t* __restrict__ tkeys, int64_t M,
                                int* __restrict__ tfirst, int* __restrict__ tcount)
{
    const int64_t n_nodes = dcount(d_nn, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const int shift = 2 * (ORDER_MAX - level[i]);
        const uint64_t lo = prefix[i] << shift, hi = (prefix[i] + 1ull) << shift;
        const int64_t a = lower_bound_u64(tkeys, 0, M, lo);
        const int64_t b = lower_bound_u64(tkeys, a, M, hi);
        tfirst[i] = (int)a;
        tcount[i] = (int)(b - a);
    }
}

// flags over the whole capacity n_cap (zero beyond the node count)
__global__ void k_collect_leaves(int n_cap, const int64_t* d_nn, const int* __restrict__ child0,
                                 const int* __restrict__ cnt, int64_t* __restrict__ flags)
{
    const int64_t nn = dcount(d_nn, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cap; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i < nn && child0[i] < 0 && cnt[i] > 0) ? 1 : 0;
}

__global__ void k_compact(int n, const int64_t* __restrict__ flags, const int64_t* __restrict__ pos, int* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i]) out[pos[i]] = (int)i;
}

inline unsigned grid_for(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

}  // namespace

// Build the tree from the key-sorted source keys.  Grows the plan's node arrays
// as needed; fills plan->level_start and plan->n_nodes.  Synchronises the
// stream once per level (the next level's size is needed on the host).
//
// Graph mode (plan->gm): no synchronisation.  Every level up to the plan's level
// capacity is launched with grids sized by the level-width capacity; the level
// bounds and the node count live in the plan's DevCounts (k_level_end), and a
// tree that would not fit (more nodes, a wider level, or a split at the last
// level) sets the overflow flag.  plan->n_nodes is the node capacity.
cudaError_t build_tree(sfmm_plan_s* P, const uint64_t* keys, int64_t n, int m, int max_depth)
{
    cudaStream_t s = P->stream;
    cudaError_t e;
    auto grow = [&](int64_t need) -> cudaError_t {
        if (need <= P->node_cap) return cudaSuccess;
        int64_t cap = need + need / 2 + 1024;
        size_t keep = (size_t)P->n_nodes;
        cudaError_t r;
        if ((r = ensure_keep(P->n_prefix, cap * 8, keep * 8, s))) return r;
        if ((r = ensure_keep(P->n_level, cap * 4, keep * 4, s))) return r;
        if ((r = ensure_keep(P->n_first, cap * 4, keep * 4, s))) return r;
        if ((r = ensure_keep(P->n_count, cap * 4, keep * 4, s))) return r;
        if ((r = ensure_keep(P->n_child0, cap * 4, keep * 4, s))) return r;
        if ((r = ensure_keep(P->n_parent, cap * 4, keep * 4, s))) return r;
        P->node_cap = cap;
        return cudaSuccess;
    };
    if (P->gm) {
        DevCounts* dc = P->dcnt.as<DevCounts>();
        const int64_t width = P->cap.width, levels = P->cap.levels;
        if ((e = grow(P->cap.nodes)) || (e = ensure(P->flags, (size_t)width * 8)) ||
            (e = ensure(P->pos, (size_t)width * 8)) || (e = ensure(P->tmp, scan_tmp_bytes(width))))
            return e;
        int64_t* flags = P->flags.as<int64_t>();
        int64_t* pos = P->pos.as<int64_t>();
        int64_t* total = P->small.as<int64_t>();
        k_level0<<<1, 32, 0, s>>>(keys, n, P->n_prefix.as<uint64_t>(), P->n_level.as<int>(), P->n_first.as<int>(),
                                  P->n_count.as<int>(), P->n_child0.as<int>(), P->n_parent.as<int>()); count_launch();
        k_counts_init<<<1, 32, 0, s>>>(dc); count_launch();
        for (int lvl = 0; lvl < levels; ++lvl) {
            k_split_flags<<<grid_for(width), 256, 0, s>>>(P->n_count.as<int>(), 0, 0, lvl, m, max_depth, flags, dc,
                                                           width); count_launch();
            if ((e = exclusive_scan_i64(flags, pos, width, total, P->tmp.p, s))) return e;
            k_level_end<<<1, 1, 0, s>>>(dc, lvl, total, P->cap.nodes, lvl == levels - 1); count_launch();
            if (lvl < levels - 1) {
                k_make_children<<<grid_for(width), 256, 0, s>>>(keys, 0, 0, lvl, flags, pos, P->n_prefix.as<uint64_t>(),
                                                               P->n_level.as<int>(), P->n_first.as<int>(),
                                                               P->n_count.as<int>(), P->n_child0.as<int>(),
                                                               P->n_parent.as<int>(), dc); count_launch();
            }
        }
        P->n_nodes = P->cap.nodes;
        return cudaGetLastError();
    }
    P->n_nodes = 0;
    if ((e = grow(12 + 4 * 1024))) return e;
    k_level0<<<1, 32, 0, s>>>(keys, n, P->n_prefix.as<uint64_t>(), P->n_level.as<int>(), P->n_first.as<int>(),
                              P->n_count.as<int>(), P->n_child0.as<int>(), P->n_parent.as<int>()); count_launch();
    P->n_nodes = 12;
    P->level_start.assign(1, 0);
    P->level_start.push_back(12);
    int lvl = 0;
    int64_t max_width = 12;
    while (true) {
        const int a = P->level_start[lvl], b = P->level_start[lvl + 1];
        const int width = b - a;
        if (width == 0 || lvl >= max_depth) break;
        max_width = std::max<int64_t>(max_width, width);
        if ((e = ensure(P->flags, (size_t)width * 8))) return e;
        if ((e = ensure(P->pos, (size_t)width * 8))) return e;
        if ((e = ensure(P->tmp, scan_tmp_bytes(width)))) return e;
        int64_t* flags = P->flags.as<int64_t>();
        int64_t* pos = P->pos.as<int64_t>();
        k_split_flags<<<grid_for(width), 256, 0, s>>>(P->n_count.as<int>(), a, b, lvl, m, max_depth, flags, nullptr,
                                                       0); count_launch();
        int64_t* total = P->small.as<int64_t>();
        if ((e = exclusive_scan_i64(flags, pos, width, total, P->tmp.p, s))) return e;
        int64_t splits = 0;
        if ((e = cudaMemcpyAsync(&splits, total, 8, cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        if (splits == 0) break;
        if ((e = grow(b + 4 * splits))) return e;
        k_make_children<<<grid_for(width), 256, 0, s>>>(keys, a, b, lvl, flags, pos, P->n_prefix.as<uint64_t>(),
                                                       P->n_level.as<int>(), P->n_first.as<int>(),
                                                       P->n_count.as<int>(), P->n_child0.as<int>(),
                                                       P->n_parent.as<int>(), nullptr); count_launch();
        P->n_nodes = b + 4 * splits;
        P->level_start.push_back((int)P->n_nodes);
        ++lvl;
    }
    P->last_max_width = max_width;
    return cudaGetLastError();
}

cudaError_t tree_geometry(sfmm_plan_s* P)
{
    cudaError_t e;
    const int64_t nn = P->n_nodes;
    if ((e = ensure(P->n_geom, (size_t)nn * GEOM_STRIDE * 8))) return e;
    k_geometry<<<grid_for(nn), 256, 0, P->stream>>>((int)nn, P->gm ? &P->dcnt.as<DevCounts>()->nn : nullptr,
                                                    P->n_prefix.as<uint64_t>(), P->n_level.as<int>(),
                                                    P->n_geom.as<double>()); count_launch();
    return cudaGetLastError();
}

cudaError_t tree_target_ranges(sfmm_plan_s* P, const uint64_t* tkeys, int64_t M)
{
    cudaError_t e;
    const int64_t nn = P->n_nodes;
    if ((e = ensure(P->n_tfirst, (size_t)nn * 4))) return e;
    if ((e = ensure(P->n_tcount, (size_t)nn * 4))) return e;
    k_target_ranges<<<grid_for(nn), 256, 0, P->stream>>>((int)nn, P->gm ? &P->dcnt.as<DevCounts>()->nn : nullptr,
                                                         P->n_prefix.as<uint64_t>(), P->n_level.as<int>(), tkeys, M,
                                                         P->n_tfirst.as<int>(), P->n_tcount.as<int>()); count_launch();
    return cudaGetLastError();
}

// Indices of the leaves whose `cnt` (source or target count) is positive.  Graph
// mode: the count goes to *d_out on the device (no synchronisation).
cudaError_t collect_leaves(sfmm_plan_s* P, const int* cnt, sfmm::Buf& out, int64_t* n_out, int64_t* d_out)
{
    cudaError_t e;
    const int64_t nn = P->n_nodes;
    cudaStream_t s = P->stream;
    if ((e = ensure(P->flags, (size_t)nn * 8))) return e;
    if ((e = ensure(P->pos, (size_t)nn * 8))) return e;
    if ((e = ensure(P->tmp, scan_tmp_bytes(nn)))) return e;
    if ((e = ensure(out, (size_t)nn * 4))) return e;
    const int64_t* d_nn = P->gm ? &P->dcnt.as<DevCounts>()->nn : nullptr;
    k_collect_leaves<<<grid_for(nn), 256, 0, s>>>((int)nn, d_nn, P->n_child0.as<int>(), cnt, P->flags.as<int64_t>()); count_launch();
    int64_t* total = P->gm ? d_out : P->small.as<int64_t>() + 1;
    if ((e = exclusive_scan_i64(P->flags.as<int64_t>(), P->pos.as<int64_t>(), nn, total, P->tmp.p, s))) return e;
    k_compact<<<grid_for(nn), 256, 0, s>>>((int)nn, P->flags.as<int64_t>(), P->pos.as<int64_t>(), out.as<int>()); count_launch();
    if (P->gm) {
        *n_out = nn;          // the capacity: launches over the leaves read *d_out
        return cudaGetLastError();
    }
    if ((e = cudaMemcpyAsync(n_out, total, 8, cudaMemcpyDeviceToHost, s))) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace sfmm
