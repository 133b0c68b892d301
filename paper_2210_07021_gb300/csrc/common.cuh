// Internal declarations shared by the CUDA translation units of libsfmm.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/sfmm.h"

namespace sfmm {

constexpr int ORDER_MAX = 29;          // r_max of Sec. 3.1
constexpr int PMAX = 32;               // largest truncation order (one coefficient per lane)
constexpr int EXP_STRIDE = 2 * PMAX + 2;   // doubles per expansion: C, Q, (Re, Im) A_1..A_PMAX
constexpr int GEOM_STRIDE = 12;        // centre(3) e_theta(3) e_phi(3) R r pad
constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ complex
struct cd { double x, y; };
__host__ __device__ __forceinline__ cd mk(double x, double y) { cd r; r.x = x; r.y = y; return r; }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ cd cscale(cd a, double s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cd cconj(cd a) { return mk(a.x, -a.y); }

// ---------------------------------------------------------- launch counting
// Every kernel launch of the library bumps this counter (reported per solve in
// sfmm_stats.launches).
void count_launch(int n = 1);
int64_t launch_total();

// ------------------------------------------------------------ device buffers
struct Buf {
    void* p = nullptr;
    size_t cap = 0;
    template <typename T> T* as() const { return static_cast<T*>(p); }
};
// Grow b to at least `bytes` (contents dropped).  Returns cudaSuccess or the error.
cudaError_t ensure(Buf& b, size_t bytes);
// Grow b to at least `bytes`, keeping the first `keep` bytes (copied on `s`).
cudaError_t ensure_keep(Buf& b, size_t bytes, size_t keep, cudaStream_t s);
void release(Buf& b);

// ------------------------------------------------------------------- scans
// Exclusive prefix sums on the device.  `tmp` must hold scan_tmp_bytes(n)
// bytes; if `total` is non-null the sum of all n inputs is written there.
size_t scan_tmp_bytes(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* tmp, cudaStream_t s);

// ------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, value) by the low `bits` bits of the key.
// The sorted data ends in (k1, v1) if *in_alt is false, else in (k2, v2).
size_t radix_tmp_bytes(int64_t n);
cudaError_t radix_sort(uint64_t* k1, uint32_t* v1, uint64_t* k2, uint32_t* v2, int64_t n, int bits,
                       void* tmp, cudaStream_t s, bool* in_alt);

// ------------------------------------------------------------------- keys
cudaError_t launch_keys(const double* xyz, int64_t n, uint64_t* keys, uint32_t* iota, cudaStream_t s);

// ------------------------------------------------------ expansion storage
// Number format of the expansions and translations: FP64, FP32 (mixed path)
// or double-float pairs of FP32 (1e-10 mixed path).
enum { EXP_F64 = 0, EXP_F32 = 1, EXP_DF = 2 };
// the parts launch_eval32 / launch_eval_df launch: the near-field kernel, the
// double-float finish (L2P and the combination, one thread per target)
enum { EVAL_NEAR = 1, EVAL_FINISH = 2 };

// --------------------------------------------------------------- the tree
struct TreeView {
    int n_nodes;          // node count, or the node capacity when d_nn is set (graph mode)
    const int64_t* d_nn;  // graph mode: the node count on the device (kernels read it there), else NULL
    const int64_t* d_level;  // graph mode: the level starts on the device (DevCounts::level), else NULL
    const uint64_t* prefix;
    const int* level;
    const int* first;     // range in key-sorted sources
    const int* count;
    const int* child0;    // -1 for a leaf
    const int* parent;    // -1 for a base box
    const double* geom;   // [node][GEOM_STRIDE]
    const int* tfirst;    // range in key-sorted targets
    const int* tcount;
};

// A count kept on the device in graph mode (d != NULL), clamped to the capacity h
// the launch was sized for; else the host value h.
__device__ __forceinline__ int64_t dcount(const int64_t* d, int64_t h)
{
    if (!d) return h;
    const int64_t v = *d;
    return v < h ? v : h;
}

// The counts of a solve run without host synchronisation (graph mode): launches
// are sized by the plan's capacities and every kernel reads its actual count
// here; a kernel that would exceed a capacity sets `overflow` instead of
// writing, and the host discards such a solve.
struct DevCounts {
    int64_t nn;             // nodes
    int64_t n_leaves;       // source leaves (count > 0)
    int64_t n_leaves_tgt;   // target leaves (tcount > 0)
    int64_t overflow;       // nonzero: a capacity was exceeded
    int64_t level[32];      // level starts: nodes of level l are [level[l], level[l + 1])
};

}  // namespace sfmm

namespace sfmm {
struct GraphState;
void graph_release(sfmm_plan_s* P);
}  // namespace sfmm

// --------------------------------------------------------------- the plan
struct sfmm_plan_s {
    int max_depth = 29;
    int p = 16;
    double tol = 0;
    sfmm_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;            // target keys + sort run here, overlapping the source tree
    bool owns_stream = false;              // a batch lane's own stream (destroyed with the plan)
    std::vector<sfmm_plan_s*> lanes;       // batch lanes: solvers on their own streams
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_m2l = nullptr;          // the M2L list is sorted (recorded by build_lists)
    cudaEvent_t ev_near[2] = {nullptr, nullptr};   // timing: around the 1e-6 path's near-field kernel
    bool forked = false;                   // the next solve finds the auxiliary stream already forked
                                           // (the host entry point copies the targets there)
    std::string err;
    int timing = 0;                        // 0 off, 1 phase times, 2 also the near-field pair count
    int* h_status = nullptr;               // pinned host word: the tensor-core M2L's status of the last solve
    // graph mode: the solve runs without host synchronisation, its launches sized by
    // these capacities and its counts kept in dcnt (DevCounts)
    bool gm = false;
    struct Caps {
        int64_t nodes = 0, width = 0, levels = 0, m2l = 0, p2p = 0, front = 0;
    } cap;
    sfmm::Buf dcnt;
    sfmm::Buf nfbuf, tleaf;                // 1e-6 path: near-field sums and leaf per sorted target
    int64_t last_max_width = 0;            // widest tree level of the last synchronised solve
    sfmm::GraphState* graph = nullptr;     // graph-launched shells (graph.cu), or NULL
    sfmm_stats stats{};

    // sources (key-sorted)
    sfmm::Buf skeys, skeys2, sperm, sperm2, src4;
    // targets (key-sorted)
    sfmm::Buf tkeys, tkeys2, tperm, tperm2, tgt4;
    // host-array staging for sfmm_deflection_host
    sfmm::Buf h_src, h_q, h_tgt, h_psi, h_alpha;
    // scratch
    sfmm::Buf tmp, flags, pos, small;   // small: a few int64 counters (device)
    sfmm::Buf ttmp;                     // scratch of the target sort (auxiliary stream)
    // tree (node arrays)
    sfmm::Buf n_prefix, n_level, n_first, n_count, n_child0, n_parent, n_geom, n_tfirst, n_tcount;
    int64_t node_cap = 0;
    std::vector<int> level_start;      // host copy: nodes of level l are [level_start[l], level_start[l+1])
    int64_t n_nodes = 0;
    // expansions
    sfmm::Buf mpole, local, tables;
    sfmm::Buf m2l_geo, m2m_geo, l2l_geo;   // translation parameters per M2L pair / per child
    sfmm::Buf soff;                        // FP32 (hi, lo) source offsets from their leaf centres (mixed path)
    sfmm::Buf toff, dc;                    // FP32 (hi, lo) target offsets and near-leaf centre offsets
    sfmm::Buf leftover;                    // M2L pairs left to the warp kernel (centres near antipodes)
    sfmm::Buf m2l_acc;                     // FP64 M2L sums per box (double-float paths)
    sfmm::Buf framedf;                     // double-float frame vectors and scale per node (double-float paths)
    sfmm::Buf dip4, adj_h, adj_g;          // adjoint: key-sorted dipoles; charges and dipoles in caller order
    sfmm::Buf logtab;                      // double-float evaluation: log(1 + j/128), 128/(128 + j), log 2
    sfmm::Buf geom32;                      // FP32 frame vectors and scale per node (mixed path)
    sfmm::Buf macn;                        // per-node sin/cos of the radii for the MAC
    sfmm::Buf macn32;                      // the same in FP32 with the centre as (hi, lo) pairs (first decision)
    // lists
    sfmm::Buf fa, fb, act, c_next, c_m2l, c_p2p, o_next, o_m2l, o_p2p;
    sfmm::Buf m2l_t, m2l_s, m2l_t2, m2l_s2, p2p_t, p2p_s, p2p_t2, p2p_s2, m2l_off, p2p_off;
    int64_t n_m2l = 0, n_p2p = 0;          // pair counts (graph mode: the list capacities)
    const int64_t* d_m2l = nullptr;        // graph mode: the pair counts on the device, else NULL
    const int64_t* d_p2p = nullptr;
    int64_t walk_cap_front = 0, walk_cap_m2l = 0, walk_cap_p2p = 0;   // list capacities that sufficed last time
    bool m2l_alt = false, p2p_alt = false;
    // node work lists
    sfmm::Buf leaves_src, leaves_tgt;
    int64_t n_leaves = 0, n_leaves_tgt = 0;
    bool skeys_alt = false, tkeys_alt = false;
    int64_t last_N = 0, last_M = 0;
};
