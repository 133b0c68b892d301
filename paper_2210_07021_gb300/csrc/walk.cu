// Interaction lists by Algorithm 1 (Sec. 3.4) with the MAC of Sec. 3.5
// (evaluated on chords, see MacNode).
//
// The recursion INTERACTION(B_S, B_T) is run breadth-first over a frontier of
// box pairs, starting from the 144 pairs of base boxes (the children of the
// root, which is the first call's B_S == B_T case).  Each round classifies
// every pair, exactly as the algorithm branches:
//   B_S == B_T, not a leaf  -> its 16 child pairs
//   B_S == B_T, a leaf      -> direct-act (P2P) of the leaf on itself
//   far (MAC1 and MAC2)     -> FMM-act (M2L)
//   neither a leaf          -> split the source if r(B_S) > r(B_T), else the target
//                              (radii equal to 1e-12 relative count as equal)
//   only the target a leaf  -> split the source; only the source a leaf -> split the target
//   both leaves             -> direct-act (P2P)
// and writes the new frontier and the two action lists at scanned offsets, so
// the output order is deterministic.  Pairs whose source box holds no
// particle, or whose target box holds no target point, are dropped (they
// contribute nothing).  The lists are then grouped by target box with a stable
// radix sort, giving CSR offsets per box.
//
// A round is three launches: classify (+ per-tile sums of the three output
// counts), a single-CTA scan of the tile sums that also advances the running
// list totals and checks capacities, and emit (in-tile scan + scatter).  The
// frontier size lives on the device, so the rounds run back to back without
// host synchronisation; 2 * depth + 4 rounds always suffice (every split makes
// one side, or for B_S == B_T both, one level deeper).  If an output would
// exceed its buffer, an overflow flag is set, nothing more is written, and the
// host grows the buffers and runs the walk again.
#include "common.cuh"

namespace sfmm {

cudaError_t radix_sort(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, int, void*, cudaStream_t, bool*);

namespace {

// Radii within this relative difference count as equal, and then the target is
// split: boxes related by a HEALPix symmetry have equal radii whose computed
// values differ only by rounding, so the comparison must not depend on it.
constexpr double RADIUS_TIE = 1e-12;

enum : uint8_t { A_DROP = 0, A_SELF = 1, A_LEAFSELF = 2, A_M2L = 3, A_SPLIT_S = 4, A_SPLIT_T = 5, A_P2P = 6 };

constexpr int WT = 256, WI = 8, WTILE = WT * WI;

// device counters (in the plan's small buffer, int64 slots)
enum { C_FRONT0 = 0, C_FRONT1 = 1, C_M2L = 2, C_P2P = 3, C_OVERFLOW = 4, C_ROUNDS = 5 };

struct WalkCaps {
    int64_t front, m2l, p2p;
};

// Per node, for the MAC without inverse trigonometry: sin and cos of R/2 and
// of c_s R/2, 2 sin(R / (2 c_t)) (3 when R / c_t >= pi: MAC2 cannot hold).
// With the chord k = |c_S - c_T| = 2 sin(d/2), monotone in d on [0, pi]:
//   MAC1  d > R_T + c_s R_S  <=>  R_T + c_s R_S < pi  and  k > 2 sin((R_T + c_s R_S)/2)
//   MAC2  d > R_T / c_t      <=>  k > 2 sin(R_T / (2 c_t))
// and, with the Near Particle Model (particles of angular radius sigma > 0),
//   MAC3  d > R_T + R_S + sigma  <=>  R_T + R_S + sigma < pi  and
//         k > 2 sin((R_T + R_S + sigma)/2),  from sin/cos of (R_S + sigma)/2:
// no particle's profile reaches a target box it acts on by M2L.
struct __align__(16) MacNode {
    double s1, c1, s2, c2, t2, R, s3, c3;
};

// FP32 copy for the walk's first decision: centre as (hi, lo) pairs (so that
// centre differences keep their relative accuracy), sines and cosines,
// counts and the first child, in one 64-byte record.
struct __align__(64) MacNode32 {
    float hx, hy, hz, lx, ly, lz, s1, c1, s2, c2, t2, R;
    int count, tcount, child0, pad;
};

__global__ void k_mac_nodes(TreeView T, double c_s, double c_t, double sigma, MacNode* __restrict__ out,
                            MacNode32* __restrict__ out32)
{
    const int64_t nn = dcount(T.d_nn, T.n_nodes);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const double R = T.geom[(size_t)i * GEOM_STRIDE + 9];
        MacNode m;
        sincos(0.5 * R, &m.s1, &m.c1);
        sincos(0.5 * c_s * R, &m.s2, &m.c2);
        const double a = R / c_t;
        m.t2 = a < 3.141592653589793 ? 2.0 * sin(0.5 * a) : 3.0;
        m.R = R;
        sincos(0.5 * (R + sigma), &m.s3, &m.c3);
        out[i] = m;
        const double* g = T.geom + (size_t)i * GEOM_STRIDE;
        MacNode32 f;
        f.hx = (float)g[0]; f.hy = (float)g[1]; f.hz = (float)g[2];
        f.lx = (float)(g[0] - (double)f.hx); f.ly = (float)(g[1] - (double)f.hy); f.lz = (float)(g[2] - (double)f.hz);
        f.s1 = (float)m.s1; f.c1 = (float)m.c1; f.s2 = (float)m.s2; f.c2 = (float)m.c2;
        f.t2 = (float)m.t2; f.R = (float)R;
        f.count = T.count[i]; f.tcount = T.tcount[i]; f.child0 = T.child0[i]; f.pad = 0;
        out32[i] = f;
    }
}

__device__ __forceinline__ uint8_t classify64(const TreeView& T, const MacNode* __restrict__ mac, int s, int t,
                                              double c_s, double sigma)
{
    if (T.count[s] == 0 || T.tcount[t] == 0) return A_DROP;
    const bool ls = T.child0[s] < 0, lt = T.child0[t] < 0;
    if (s == t) return ls ? A_LEAFSELF : A_SELF;
    const double* gs = T.geom + (size_t)s * GEOM_STRIDE;
    const double* gt = T.geom + (size_t)t * GEOM_STRIDE;
    const double dx = gs[0] - gt[0], dy = gs[1] - gt[1], dz = gs[2] - gt[2];
    const double k2 = dx * dx + dy * dy + dz * dz;
    const MacNode ms = mac[s], mt = mac[t];
    const double Rs = ms.R, Rt = mt.R;
    const double thr1 = 2.0 * (mt.s1 * ms.c2 + mt.c1 * ms.s2);
    const bool mac1 = (Rt + c_s * Rs < 3.141592653589793) && k2 > thr1 * thr1;
    const bool mac2 = k2 > mt.t2 * mt.t2;
    bool mac3 = true;
    if (sigma > 0.0) {
        const double thr3 = 2.0 * (mt.s1 * ms.c3 + mt.c1 * ms.s3);
        mac3 = (Rt + Rs + sigma < 3.141592653589793) && k2 > thr3 * thr3;
    }
    if (mac1 && mac2 && mac3) return A_M2L;
    if (!ls && !lt) return (Rs > Rt * (1.0 + RADIUS_TIE)) ? A_SPLIT_S : A_SPLIT_T;
    if (!ls) return A_SPLIT_S;
    if (!lt) return A_SPLIT_T;
    return A_P2P;
}

// The decision of classify64, taken in FP32 when every comparison it rests on
// has a relative margin of at least 1e-5 (the FP32 quantities are accurate to
// a few 1e-7: centre differences from (hi, lo) pairs, rounded sines and
// cosines), else by classify64 itself, so the outcome is classify64's.  The
// classification is otherwise bound by the FP64 pipe, which this GPU runs at
// 1/64 of the FP32 rate.
__device__ __forceinline__ uint8_t classify(const TreeView& T, const MacNode* __restrict__ mac,
                                            const MacNode32* __restrict__ mac32, int s, int t, double c_s,
                                            double sigma)
{
    const MacNode32 a = mac32[s], b = mac32[t];
    if (a.count == 0 || b.tcount == 0) return A_DROP;
    const bool ls = a.child0 < 0, lt = b.child0 < 0;
    if (s == t) return ls ? A_LEAFSELF : A_SELF;
    if (sigma > 0.0) return classify64(T, mac, s, t, c_s, sigma);
    constexpr float EPS = 1e-5f;
    const float dx = (a.hx - b.hx) + (a.lx - b.lx), dy = (a.hy - b.hy) + (a.ly - b.ly), dz = (a.hz - b.hz) + (a.lz - b.lz);
    const float k2 = dx * dx + dy * dy + dz * dz;
    const float thr1 = 2.f * (b.s1 * a.c2 + b.c1 * a.s2);
    const float th2 = thr1 * thr1, t22 = b.t2 * b.t2;
    const float sum1 = b.R + (float)c_s * a.R;
    const float pi = 3.14159265f;
    if (fabsf(k2 - th2) <= EPS * (k2 + th2) || fabsf(k2 - t22) <= EPS * (k2 + t22) || fabsf(sum1 - pi) <= EPS * pi)
        return classify64(T, mac, s, t, c_s, sigma);
    if (sum1 < pi && k2 > th2 && k2 > t22) return A_M2L;
    if (!ls && !lt) {
        if (fabsf(a.R - b.R) <= EPS * b.R) return classify64(T, mac, s, t, c_s, sigma);
        return a.R > b.R ? A_SPLIT_S : A_SPLIT_T;
    }
    if (!ls) return A_SPLIT_S;
    if (!lt) return A_SPLIT_T;
    return A_P2P;
}

__device__ __forceinline__ int3 counts_of(uint8_t a)
{
    return make_int3((a == A_SELF) ? 16 : ((a == A_SPLIT_S || a == A_SPLIT_T) ? 4 : 0), (a == A_M2L) ? 1 : 0,
                     (a == A_P2P || a == A_LEAFSELF) ? 1 : 0);
}

__device__ __forceinline__ int3 add3(int3 a, int3 b) { return make_int3(a.x + b.x, a.y + b.y, a.z + b.z); }

__device__ __forceinline__ int3 warp_incl3(int3 v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(FULL, v.x, o), y = __shfl_up_sync(FULL, v.y, o), z = __shfl_up_sync(FULL, v.z, o);
        if (lane >= o) { v.x += x; v.y += y; v.z += z; }
    }
    return v;
}

// block (256 threads) exclusive scan of one int3 per thread; *total = block sum
__device__ __forceinline__ int3 block_excl3(int3 v, int3* s_w, int3* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int3 inc = warp_incl3(v, lane);
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        int3 x = lane < (WT / 32) ? s_w[lane] : make_int3(0, 0, 0);
        const int3 xi = warp_incl3(x, lane);
        if (lane < (WT / 32)) s_w[lane] = make_int3(xi.x - x.x, xi.y - x.y, xi.z - x.z);
        if (lane == (WT / 32) - 1) *total = xi;
    }
    __syncthreads();
    const int3 wb = s_w[w];
    return make_int3(inc.x - v.x + wb.x, inc.y - v.y + wb.y, inc.z - v.z + wb.z);
}

__global__ void k_init_frontier(int2* f, int64_t* ctr)
{
    const int i = threadIdx.x;
    if (i < 144) f[i] = make_int2(i / 12, i % 12);
    if (i == 0) {
        ctr[C_FRONT0] = 144;
        ctr[C_FRONT1] = 0;
        ctr[C_M2L] = 0;
        ctr[C_P2P] = 0;
        ctr[C_OVERFLOW] = 0;
        ctr[C_ROUNDS] = 0;
    }
}

__global__ void __launch_bounds__(WT) k_walk_classify(TreeView T, const MacNode* __restrict__ mac,
                                                      const MacNode32* __restrict__ mac32,
                                                      const int2* __restrict__ front,
                                                      const int64_t* __restrict__ n_front_p, double c_s, double sigma,
                                                      uint8_t* __restrict__ act, int3* __restrict__ tile_sums)
{
    __shared__ int3 s_w[WT / 32];
    __shared__ int3 s_tot;
    const int64_t n = *n_front_p;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int3 acc = make_int3(0, 0, 0);
        for (int r = 0; r < WI; ++r) {
            const int64_t i = tile * WTILE + (int64_t)r * WT + threadIdx.x;
            if (i < n) {
                const int2 pr = front[i];
                const uint8_t a = classify(T, mac, mac32, pr.x, pr.y, c_s, sigma);
                act[i] = a;
                acc = add3(acc, counts_of(a));
            }
        }
        block_excl3(acc, s_w, &s_tot);
        if (threadIdx.x == 0) tile_sums[tile] = s_tot;
        __syncthreads();
    }
}

// single CTA: exclusive scan of the tile sums; bases of this round's outputs
__global__ void __launch_bounds__(WT) k_walk_top(int3* __restrict__ tile_sums, const int64_t* __restrict__ n_front_p,
                                                 int64_t* __restrict__ n_next_p, int64_t* __restrict__ ctr,
                                                 int64_t* __restrict__ bases, WalkCaps caps)
{
    __shared__ int3 s_w[WT / 32];
    __shared__ int3 s_tot;
    const int64_t n = *n_front_p;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    int64_t cx = 0, cy = 0, cz = 0;
    for (int64_t c0 = 0; c0 < ntiles; c0 += WT) {
        const int64_t e = c0 + threadIdx.x;
        const int3 v = e < ntiles ? tile_sums[e] : make_int3(0, 0, 0);
        const int3 ex = block_excl3(v, s_w, &s_tot);
        // tile offsets fit in int: a round's outputs are far below 2^31
        if (e < ntiles) tile_sums[e] = make_int3((int)(ex.x + cx), (int)(ex.y + cy), (int)(ex.z + cz));
        cx += s_tot.x; cy += s_tot.y; cz += s_tot.z;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t m0 = ctr[C_M2L], p0 = ctr[C_P2P];
        bases[0] = m0;
        bases[1] = p0;
        if (cx > caps.front || m0 + cy > caps.m2l || p0 + cz > caps.p2p || ctr[C_OVERFLOW]) {
            ctr[C_OVERFLOW] = 1;
            *n_next_p = 0;            // stop the walk; the host grows the buffers and reruns it
            bases[2] = 1;
        } else {
            ctr[C_M2L] = m0 + cy;
            ctr[C_P2P] = p0 + cz;
            *n_next_p = cx;
            bases[2] = 0;
        }
        ctr[C_ROUNDS] += 1;
    }
}

__global__ void __launch_bounds__(WT) k_walk_emit(TreeView T, const int2* __restrict__ front,
                                                  const int64_t* __restrict__ n_front_p, const uint8_t* __restrict__ act,
                                                  const int3* __restrict__ tile_off, const int64_t* __restrict__ bases,
                                                  int2* __restrict__ next, uint64_t* __restrict__ m2l_t,
                                                  uint32_t* __restrict__ m2l_s, uint64_t* __restrict__ p2p_t,
                                                  uint32_t* __restrict__ p2p_s)
{
    __shared__ int3 s_w[WT / 32];
    __shared__ int3 s_tot;
    __shared__ uint8_t s_act[WTILE];
    if (bases[2]) return;         // overflow: write nothing
    const int64_t n = *n_front_p;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    const int64_t mb = bases[0], pb = bases[1];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * WTILE;
        for (int r = 0; r < WI; ++r) {
            const int64_t i = t0 + (int64_t)r * WT + threadIdx.x;
            s_act[r * WT + threadIdx.x] = i < n ? act[i] : A_DROP;
        }
        __syncthreads();
        // thread-local run of WI consecutive items (blocked), then a block scan
        int3 loc[WI];
        int3 acc = make_int3(0, 0, 0);
        for (int r = 0; r < WI; ++r) {
            loc[r] = acc;
            acc = add3(acc, counts_of(s_act[threadIdx.x * WI + r]));
        }
        const int3 ex = block_excl3(acc, s_w, &s_tot);
        const int3 to = tile_off[tile];
        for (int r = 0; r < WI; ++r) {
            const int64_t i = t0 + (int64_t)threadIdx.x * WI + r;
            if (i >= n) break;
            const uint8_t a = s_act[threadIdx.x * WI + r];
            if (a == A_DROP) continue;
            const int2 pr = front[i];
            const int s = pr.x, t = pr.y;
            const int64_t on = (int64_t)to.x + ex.x + loc[r].x;
            if (a == A_SELF) {
                const int c = T.child0[s];
                int2* o = next + on;
                for (int u = 0; u < 4; ++u)
                    for (int v = 0; v < 4; ++v) o[u * 4 + v] = make_int2(c + u, c + v);
            } else if (a == A_SPLIT_S) {
                const int c = T.child0[s];
                for (int u = 0; u < 4; ++u) next[on + u] = make_int2(c + u, t);
            } else if (a == A_SPLIT_T) {
                const int c = T.child0[t];
                for (int u = 0; u < 4; ++u) next[on + u] = make_int2(s, c + u);
            } else if (a == A_M2L) {
                const int64_t om = mb + to.y + ex.y + loc[r].y;
                m2l_t[om] = (uint64_t)t;
                m2l_s[om] = (uint32_t)s;
            } else {
                const int64_t op = pb + to.z + ex.z + loc[r].z;
                p2p_t[op] = (uint64_t)t;
                p2p_s[op] = (uint32_t)s;
            }
        }
        __syncthreads();
    }
}

__global__ void k_csr_offsets(const uint64_t* __restrict__ sorted_t, int64_t n_cap, const int64_t* d_np, int n_nodes,
                              int64_t* __restrict__ off)
{
    const int64_t n_pairs = dcount(d_np, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n_pairs;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (sorted_t[mid] < (uint64_t)i) lo = mid + 1; else hi = mid;
        }
        off[i] = lo;
    }
}

// Graph mode: the list entries past the walk's count get a target key that sorts
// after every node (all ones in the sorted bits), so that sorting the whole
// capacity sorts the list.
__global__ void k_pad_pairs(uint64_t* __restrict__ t, uint32_t* __restrict__ src, const int64_t* __restrict__ n,
                            int64_t cap, uint64_t key)
{
    for (int64_t i = *n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x) {
        t[i] = key;
        src[i] = 0u;
    }
}

// Graph mode: a walk that overflowed its capacities or left a frontier voids the solve.
__global__ void k_walk_check(const int64_t* __restrict__ ctr, int left_slot, DevCounts* dc)
{
    if (ctr[C_OVERFLOW] || ctr[left_slot] != 0) dc->overflow = 1;
}

inline unsigned grid_for(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

inline int bits_for(int64_t n)
{
    int b = 1;
    while (b < 63 && (int64_t(1) << b) <= n) ++b;
    return b;
}

}  // namespace

// Run Algorithm 1 and build the grouped M2L and P2P lists in the plan.
//
// Graph mode (plan->gm): no synchronisation.  The walk runs 2 (level capacity) + 4
// rounds into buffers of the plan's list capacities; the pair counts stay on the
// device (plan->d_m2l, plan->d_p2p), the entries past them are padded to sort
// last and the whole capacity is sorted; an overflow of the walk voids the solve.
cudaError_t build_lists(sfmm_plan_s* P, const TreeView& T, double c_s, double c_t, cudaStream_t s)
{
    cudaError_t e;
    const int depth = P->gm ? (int)P->cap.levels : (int)P->level_start.size() - 2;
    const int rounds = 2 * depth + 4;
    int64_t* ctr = P->small.as<int64_t>() + 24;      // [24..29] counters, [30..32] bases
    int64_t* bases = ctr + 6;
    // capacities: start from the last solve's needs, or from the node count
    int64_t cap_front = std::max<int64_t>(P->walk_cap_front, std::max<int64_t>(4096, 32 * P->n_nodes));
    int64_t cap_m2l = std::max<int64_t>(P->walk_cap_m2l, std::max<int64_t>(4096, 48 * P->n_nodes));
    int64_t cap_p2p = std::max<int64_t>(P->walk_cap_p2p, std::max<int64_t>(4096, 16 * P->n_nodes));
    if (P->gm) {
        cap_front = P->cap.front;
        cap_m2l = P->cap.m2l;
        cap_p2p = P->cap.p2p;
    }
    if ((e = ensure(P->macn, (size_t)P->n_nodes * sizeof(MacNode))) ||
        (e = ensure(P->macn32, (size_t)P->n_nodes * sizeof(MacNode32))))
        return e;
    k_mac_nodes<<<grid_for(P->n_nodes), 256, 0, s>>>(T, c_s, c_t, P->opt.sigma, P->macn.as<MacNode>(),
                                                     P->macn32.as<MacNode32>());
    count_launch();
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((e = ensure(P->fa, (size_t)cap_front * 8)) || (e = ensure(P->fb, (size_t)cap_front * 8)) ||
            (e = ensure(P->act, (size_t)cap_front)) ||
            (e = ensure(P->c_next, (size_t)((cap_front + WTILE - 1) / WTILE + 1) * sizeof(int3))) ||
            (e = ensure(P->m2l_t, (size_t)cap_m2l * 8)) || (e = ensure(P->m2l_s, (size_t)cap_m2l * 4)) ||
            (e = ensure(P->p2p_t, (size_t)cap_p2p * 8)) || (e = ensure(P->p2p_s, (size_t)cap_p2p * 4)))
            return e;
        k_init_frontier<<<1, 160, 0, s>>>(P->fa.as<int2>(), ctr); count_launch();
        WalkCaps caps{cap_front, cap_m2l, cap_p2p};
        const unsigned grid = 152 * 4;
        for (int r = 0; r < rounds; ++r) {
            const int2* front = (r & 1) ? P->fb.as<int2>() : P->fa.as<int2>();
            int2* next = (r & 1) ? P->fa.as<int2>() : P->fb.as<int2>();
            int64_t* nf = ctr + ((r & 1) ? C_FRONT1 : C_FRONT0);
            int64_t* nn = ctr + ((r & 1) ? C_FRONT0 : C_FRONT1);
            k_walk_classify<<<grid, WT, 0, s>>>(T, P->macn.as<MacNode>(), P->macn32.as<MacNode32>(), front, nf, c_s,
                                                P->opt.sigma,
                                                P->act.as<uint8_t>(),
                                                P->c_next.as<int3>());
            count_launch();
            k_walk_top<<<1, WT, 0, s>>>(P->c_next.as<int3>(), nf, nn, ctr, bases, caps); count_launch();
            k_walk_emit<<<grid, WT, 0, s>>>(T, front, nf, P->act.as<uint8_t>(), P->c_next.as<int3>(), bases, next,
                                            P->m2l_t.as<uint64_t>(), P->m2l_s.as<uint32_t>(), P->p2p_t.as<uint64_t>(),
                                            P->p2p_s.as<uint32_t>());
            count_launch();
        }
        if ((e = cudaGetLastError())) return e;
        if (P->gm) {
            k_walk_check<<<1, 1, 0, s>>>(ctr, (rounds & 1) ? C_FRONT1 : C_FRONT0, P->dcnt.as<DevCounts>()); count_launch();
            P->n_m2l = cap_m2l;
            P->n_p2p = cap_p2p;
            P->d_m2l = ctr + C_M2L;
            P->d_p2p = ctr + C_P2P;
            break;
        }
        int64_t h[6];
        if ((e = cudaMemcpyAsync(h, ctr, sizeof h, cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        const int64_t left = h[(rounds & 1) ? C_FRONT1 : C_FRONT0];
        if (!h[C_OVERFLOW] && left == 0) {
            P->n_m2l = h[C_M2L];
            P->n_p2p = h[C_P2P];
            break;
        }
        if (!h[C_OVERFLOW] && left != 0) return cudaErrorUnknown;   // cannot happen: the round bound is exact
        cap_front *= 2;
        cap_m2l *= 2;
        cap_p2p *= 2;
        if (attempt == 7) return cudaErrorMemoryAllocation;
    }
    P->walk_cap_front = cap_front;
    P->walk_cap_m2l = cap_m2l;
    P->walk_cap_p2p = cap_p2p;
    const int64_t n_m2l = P->n_m2l, n_p2p = P->n_p2p;
    // group by target box (stable), then CSR offsets
    const int bits = bits_for(P->n_nodes);
    if (P->gm) {
        const uint64_t pad = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
        k_pad_pairs<<<grid_for(n_m2l), 256, 0, s>>>(P->m2l_t.as<uint64_t>(), P->m2l_s.as<uint32_t>(), P->d_m2l, n_m2l,
                                                    pad); count_launch();
        k_pad_pairs<<<grid_for(n_p2p), 256, 0, s>>>(P->p2p_t.as<uint64_t>(), P->p2p_s.as<uint32_t>(), P->d_p2p, n_p2p,
                                                    pad); count_launch();
    } else {
        P->d_m2l = P->d_p2p = nullptr;
    }
    if ((e = ensure(P->m2l_t2, (size_t)std::max<int64_t>(n_m2l, 1) * 8)) ||
        (e = ensure(P->m2l_s2, (size_t)std::max<int64_t>(n_m2l, 1) * 4)))
        return e;
    if ((e = ensure(P->p2p_t2, (size_t)std::max<int64_t>(n_p2p, 1) * 8)) ||
        (e = ensure(P->p2p_s2, (size_t)std::max<int64_t>(n_p2p, 1) * 4)))
        return e;
    if ((e = ensure(P->tmp, radix_tmp_bytes(std::max(n_m2l, n_p2p))))) return e;
    if ((e = ensure(P->m2l_off, (size_t)(P->n_nodes + 1) * 8)) || (e = ensure(P->p2p_off, (size_t)(P->n_nodes + 1) * 8)))
        return e;
    // the M2L list first: its event (plan->ev_m2l) lets M2L start while the P2P list is sorted
    if ((e = radix_sort(P->m2l_t.as<uint64_t>(), P->m2l_s.as<uint32_t>(), P->m2l_t2.as<uint64_t>(),
                        P->m2l_s2.as<uint32_t>(), n_m2l, bits, P->tmp.p, s, &P->m2l_alt)))
        return e;
    const uint64_t* mt = P->m2l_alt ? P->m2l_t2.as<uint64_t>() : P->m2l_t.as<uint64_t>();
    k_csr_offsets<<<grid_for(P->n_nodes + 1), 256, 0, s>>>(mt, n_m2l, P->d_m2l, (int)P->n_nodes,
                                                           P->m2l_off.as<int64_t>()); count_launch();
    if ((e = cudaEventRecord(P->ev_m2l, s))) return e;
    if ((e = radix_sort(P->p2p_t.as<uint64_t>(), P->p2p_s.as<uint32_t>(), P->p2p_t2.as<uint64_t>(),
                        P->p2p_s2.as<uint32_t>(), n_p2p, bits, P->tmp.p, s, &P->p2p_alt)))
        return e;
    const uint64_t* pt = P->p2p_alt ? P->p2p_t2.as<uint64_t>() : P->p2p_t.as<uint64_t>();
    k_csr_offsets<<<grid_for(P->n_nodes + 1), 256, 0, s>>>(pt, n_p2p, P->d_p2p, (int)P->n_nodes,
                                                           P->p2p_off.as<int64_t>()); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
