// Interaction lists by Algorithm 1 (Sec. 3.4) with the MAC of Sec. 3.5.
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
#include "common.cuh"

namespace sfmm {

cudaError_t radix_sort(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, int, void*, cudaStream_t, bool*);

namespace {

// Radii within this relative difference count as equal, and then the target is
// split: boxes related by a HEALPix symmetry have equal radii whose computed
// values differ only by rounding, so the comparison must not depend on it.
constexpr double RADIUS_TIE = 1e-12;

enum : uint8_t { A_DROP = 0, A_SELF = 1, A_LEAFSELF = 2, A_M2L = 3, A_SPLIT_S = 4, A_SPLIT_T = 5, A_P2P = 6 };

__global__ void k_init_frontier(int2* f)
{
    const int i = threadIdx.x;
    if (i < 144) f[i] = make_int2(i / 12, i % 12);
}

__global__ void k_classify(TreeView T, const int2* __restrict__ front, int64_t n, double c_s, double c_t,
                           uint8_t* __restrict__ act, int64_t* __restrict__ c_next, int64_t* __restrict__ c_m2l,
                           int64_t* __restrict__ c_p2p)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = front[i].x, t = front[i].y;
        uint8_t a;
        if (T.count[s] == 0 || T.tcount[t] == 0) {
            a = A_DROP;
        } else {
            const bool ls = T.child0[s] < 0, lt = T.child0[t] < 0;
            if (s == t) {
                a = ls ? A_LEAFSELF : A_SELF;
            } else {
                const double* gs = T.geom + (size_t)s * GEOM_STRIDE;
                const double* gt = T.geom + (size_t)t * GEOM_STRIDE;
                const double dx = gs[0] - gt[0], dy = gs[1] - gt[1], dz = gs[2] - gt[2];
                const double d = 2.0 * asin(fmin(1.0, 0.5 * sqrt(dx * dx + dy * dy + dz * dz)));
                const double Rs = gs[9], Rt = gt[9];
                if (d - Rt - c_s * Rs > 0.0 && Rt < c_t * d) a = A_M2L;
                else if (!ls && !lt) a = (Rs > Rt * (1.0 + RADIUS_TIE)) ? A_SPLIT_S : A_SPLIT_T;
                else if (!ls) a = A_SPLIT_S;
                else if (!lt) a = A_SPLIT_T;
                else a = A_P2P;
            }
        }
        act[i] = a;
        c_next[i] = (a == A_SELF) ? 16 : ((a == A_SPLIT_S || a == A_SPLIT_T) ? 4 : 0);
        c_m2l[i] = (a == A_M2L) ? 1 : 0;
        c_p2p[i] = (a == A_P2P || a == A_LEAFSELF) ? 1 : 0;
    }
}

__global__ void k_emit(TreeView T, const int2* __restrict__ front, int64_t n, const uint8_t* __restrict__ act,
                       const int64_t* __restrict__ o_next, const int64_t* __restrict__ o_m2l,
                       const int64_t* __restrict__ o_p2p, int2* __restrict__ next, uint64_t* __restrict__ m2l_t,
                       uint32_t* __restrict__ m2l_s, uint64_t* __restrict__ p2p_t, uint32_t* __restrict__ p2p_s)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = front[i].x, t = front[i].y;
        const uint8_t a = act[i];
        if (a == A_SELF) {
            const int c = T.child0[s];
            int2* o = next + o_next[i];
            for (int u = 0; u < 4; ++u)
                for (int v = 0; v < 4; ++v) o[u * 4 + v] = make_int2(c + u, c + v);
        } else if (a == A_SPLIT_S) {
            const int c = T.child0[s];
            int2* o = next + o_next[i];
            for (int u = 0; u < 4; ++u) o[u] = make_int2(c + u, t);
        } else if (a == A_SPLIT_T) {
            const int c = T.child0[t];
            int2* o = next + o_next[i];
            for (int u = 0; u < 4; ++u) o[u] = make_int2(s, c + u);
        } else if (a == A_M2L) {
            m2l_t[o_m2l[i]] = (uint64_t)t;
            m2l_s[o_m2l[i]] = (uint32_t)s;
        } else if (a == A_P2P || a == A_LEAFSELF) {
            p2p_t[o_p2p[i]] = (uint64_t)t;
            p2p_s[o_p2p[i]] = (uint32_t)s;
        }
    }
}

__global__ void k_csr_offsets(const uint64_t* __restrict__ sorted_t, int64_t n_pairs, int n_nodes,
                              int64_t* __restrict__ off)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n_pairs;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (sorted_t[mid] < (uint64_t)i) lo = mid + 1; else hi = mid;
        }
        off[i] = lo;
    }
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
cudaError_t build_lists(sfmm_plan_s* P, const TreeView& T, double c_s, double c_t)
{
    cudaStream_t s = P->stream;
    cudaError_t e;
    int64_t cap_front = 1 << 16, cap_m2l = 1 << 16, cap_p2p = 1 << 16;
    auto need = [&](Buf& b, int64_t bytes) { return ensure_keep(b, (size_t)bytes, 0, s); };
    if ((e = need(P->fa, cap_front * 8)) || (e = need(P->fb, cap_front * 8))) return e;
    cap_front = (int64_t)std::min(P->fa.cap, P->fb.cap) / 8;
    int64_t n_front = 144;
    int64_t n_m2l = 0, n_p2p = 0;
    k_init_frontier<<<1, 160, 0, s>>>(P->fa.as<int2>()); count_launch();
    // list storage: grown as rounds add pairs
    auto grow_list = [&](Buf& bt, Buf& bs, int64_t used, int64_t want) -> cudaError_t {
        cudaError_t r;
        if ((size_t)want * 8 > bt.cap) {
            size_t nb = (size_t)(want + want / 2 + 4096);
            if ((r = ensure_keep(bt, nb * 8, (size_t)used * 8, s))) return r;
            if ((r = ensure_keep(bs, nb * 4, (size_t)used * 4, s))) return r;
        }
        return cudaSuccess;
    };
    if ((e = grow_list(P->m2l_t, P->m2l_s, 0, cap_m2l))) return e;
    if ((e = grow_list(P->p2p_t, P->p2p_s, 0, cap_p2p))) return e;
    int64_t* totals = P->small.as<int64_t>() + 4;   // [4..6]: next, m2l, p2p
    int rounds = 0;
    while (n_front > 0) {
        if (++rounds > 4 * (ORDER_MAX + 2)) return cudaErrorUnknown;   // the recursion is at most 2 per level
        if ((e = ensure(P->act, (size_t)n_front))) return e;
        if ((e = ensure(P->c_next, (size_t)n_front * 8)) || (e = ensure(P->c_m2l, (size_t)n_front * 8)) ||
            (e = ensure(P->c_p2p, (size_t)n_front * 8)))
            return e;
        if ((e = ensure(P->o_next, (size_t)n_front * 8)) || (e = ensure(P->o_m2l, (size_t)n_front * 8)) ||
            (e = ensure(P->o_p2p, (size_t)n_front * 8)))
            return e;
        if ((e = ensure(P->tmp, scan_tmp_bytes(n_front)))) return e;
        k_classify<<<grid_for(n_front), 256, 0, s>>>(T, P->fa.as<int2>(), n_front, c_s, c_t, P->act.as<uint8_t>(),
                                                     P->c_next.as<int64_t>(), P->c_m2l.as<int64_t>(),
                                                     P->c_p2p.as<int64_t>()); count_launch();
        if ((e = exclusive_scan_i64(P->c_next.as<int64_t>(), P->o_next.as<int64_t>(), n_front, totals, P->tmp.p, s)))
            return e;
        if ((e = exclusive_scan_i64(P->c_m2l.as<int64_t>(), P->o_m2l.as<int64_t>(), n_front, totals + 1, P->tmp.p, s)))
            return e;
        if ((e = exclusive_scan_i64(P->c_p2p.as<int64_t>(), P->o_p2p.as<int64_t>(), n_front, totals + 2, P->tmp.p, s)))
            return e;
        int64_t h[3];
        if ((e = cudaMemcpyAsync(h, totals, 24, cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        if (h[0] * 8 > (int64_t)P->fb.cap) {
            if ((e = ensure(P->fb, (size_t)(h[0] + h[0] / 2 + 1024) * 8))) return e;
        }
        if ((e = grow_list(P->m2l_t, P->m2l_s, n_m2l, n_m2l + h[1]))) return e;
        if ((e = grow_list(P->p2p_t, P->p2p_s, n_p2p, n_p2p + h[2]))) return e;
        k_emit<<<grid_for(n_front), 256, 0, s>>>(T, P->fa.as<int2>(), n_front, P->act.as<uint8_t>(),
                                                 P->o_next.as<int64_t>(), P->o_m2l.as<int64_t>(),
                                                 P->o_p2p.as<int64_t>(), P->fb.as<int2>(),
                                                 P->m2l_t.as<uint64_t>() + n_m2l, P->m2l_s.as<uint32_t>() + n_m2l,
                                                 P->p2p_t.as<uint64_t>() + n_p2p, P->p2p_s.as<uint32_t>() + n_p2p); count_launch();
        if ((e = cudaGetLastError())) return e;
        n_m2l += h[1];
        n_p2p += h[2];
        std::swap(P->fa, P->fb);
        n_front = h[0];
    }
    P->n_m2l = n_m2l;
    P->n_p2p = n_p2p;
    // group by target box (stable), then CSR offsets
    const int bits = bits_for(P->n_nodes);
    if ((e = ensure(P->m2l_t2, (size_t)std::max<int64_t>(n_m2l, 1) * 8)) ||
        (e = ensure(P->m2l_s2, (size_t)std::max<int64_t>(n_m2l, 1) * 4)))
        return e;
    if ((e = ensure(P->p2p_t2, (size_t)std::max<int64_t>(n_p2p, 1) * 8)) ||
        (e = ensure(P->p2p_s2, (size_t)std::max<int64_t>(n_p2p, 1) * 4)))
        return e;
    if ((e = ensure(P->tmp, radix_tmp_bytes(std::max(n_m2l, n_p2p))))) return e;
    if ((e = radix_sort(P->m2l_t.as<uint64_t>(), P->m2l_s.as<uint32_t>(), P->m2l_t2.as<uint64_t>(),
                        P->m2l_s2.as<uint32_t>(), n_m2l, bits, P->tmp.p, s, &P->m2l_alt)))
        return e;
    if ((e = radix_sort(P->p2p_t.as<uint64_t>(), P->p2p_s.as<uint32_t>(), P->p2p_t2.as<uint64_t>(),
                        P->p2p_s2.as<uint32_t>(), n_p2p, bits, P->tmp.p, s, &P->p2p_alt)))
        return e;
    if ((e = ensure(P->m2l_off, (size_t)(P->n_nodes + 1) * 8)) || (e = ensure(P->p2p_off, (size_t)(P->n_nodes + 1) * 8)))
        return e;
    const uint64_t* mt = P->m2l_alt ? P->m2l_t2.as<uint64_t>() : P->m2l_t.as<uint64_t>();
    const uint64_t* pt = P->p2p_alt ? P->p2p_t2.as<uint64_t>() : P->p2p_t.as<uint64_t>();
    k_csr_offsets<<<grid_for(P->n_nodes + 1), 256, 0, s>>>(mt, n_m2l, (int)P->n_nodes, P->m2l_off.as<int64_t>()); count_launch();
    k_csr_offsets<<<grid_for(P->n_nodes + 1), 256, 0, s>>>(pt, n_p2p, (int)P->n_nodes, P->p2p_off.as<int64_t>()); count_launch();
    return cudaGetLastError();
}

}  // namespace sfmm
