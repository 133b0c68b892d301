// Graph-launched shells: the solves of a batch of shells (the N_L lensing
// planes of the multi-plane setting, Sec. 2.1) recorded once into one CUDA
// graph and replayed.
//
// Each shell has its own solver in graph mode: no host synchronisation inside
// the solve.  The tree levels, the list walk (Algorithm 1) and every launch over
// leaves or pairs are sized by capacities planned from a synchronised solve of
// the same shell, and read their actual counts on the device (DevCounts,
// build_tree, build_lists).  The shells' solvers run on their own streams,
// forked from and joined back into the graph's origin stream, so that the small
// launches of one shell (tree levels, walk rounds) overlap the large kernels of
// another.  After a replay the host reads every shell's overflow flag (one
// synchronisation for the whole batch): a shell whose tree or lists outgrew a
// capacity is solved again synchronously (its results replace the replay's),
// its capacities are planned anew and the graph is recorded again.
//
// Buffers are never reallocated while a graph holds them: before a recording,
// every shell's solver has run one complete graph-mode solve eagerly (which
// sizes every buffer for its capacities), so the recorded solve allocates
// nothing.
#include "common.cuh"

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

namespace sfmm {

sfmm_status solve_entry(sfmm_plan_s* P, const double* src, const void* q, int64_t N, const double* tgt, int64_t M,
                        double* psi, double* alpha);
sfmm_status plan_error(sfmm_plan_s* P, sfmm_status st, const std::string& msg);

namespace {

// pinned host copy of a shell's device counts, written by the graph's last nodes
struct ShellReport {
    DevCounts dc;
    int64_t n_m2l, n_p2p;
};

}  // namespace

struct GraphState {
    int n = 0;
    std::vector<sfmm_plan_s*> shells;      // one graph-mode solver per shell (own stream and buffers)
    std::vector<const double*> src, tgt;
    std::vector<const void*> q;
    std::vector<int64_t> N, M;
    std::vector<double*> psi, alpha;
    double slack = 0.25;
    cudaStream_t origin = nullptr;         // the stream the graph is recorded from
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_done;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ShellReport* h_rep = nullptr;          // pinned [n]
    int64_t kernel_nodes = 0, launches = 0, overflows = 0, recaptures = 0;
};

namespace {

sfmm_status cuda_err(sfmm_plan_s* P, cudaError_t e, const char* where)
{
    return plan_error(P, e == cudaErrorMemoryAllocation ? SFMM_ENOMEM : SFMM_ECUDA,
                      std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}

// Capacities of a shell's graph-mode solve from its last synchronised solve:
// each count times (1 + slack) plus a margin; one level more than the tree had
// (bounded by the depth limit), and the walk frontier the synchronised walk used.
void plan_caps(sfmm_plan_s* L, double slack)
{
    const double f = 1.0 + slack;
    const int depth = L->level_start.size() >= 2 ? (int)L->level_start.size() - 2 : 1;
    L->cap.nodes = (int64_t)((double)L->n_nodes * f) + 1024;
    L->cap.width = (int64_t)((double)L->last_max_width * f) + 256;
    L->cap.levels = std::min<int64_t>(depth + 2, (int64_t)L->max_depth + 1);
    L->cap.m2l = (int64_t)((double)L->n_m2l * f) + 4096;
    L->cap.p2p = (int64_t)((double)L->n_p2p * f) + 4096;
    L->cap.front = std::max<int64_t>(L->walk_cap_front, 32 * L->cap.nodes);
}

// A synchronised solve of shell i, then its capacities, then one eager
// graph-mode solve (which sizes every buffer); the eager solve's counts are
// checked on the host.
sfmm_status prepare_shell(sfmm_plan_s* P, GraphState* G, int i)
{
    sfmm_plan_s* L = G->shells[i];
    L->gm = false;
    sfmm_status st = solve_entry(L, G->src[i], G->q[i], G->N[i], G->tgt[i], G->M[i], G->psi[i], G->alpha[i]);
    if (st != SFMM_OK) return plan_error(P, st, "shell " + std::to_string(i) + ": " + L->err);
    plan_caps(L, G->slack);
    cudaError_t e;
    if ((e = ensure(L->dcnt, sizeof(DevCounts)))) return cuda_err(P, e, "graph counts");
    if ((e = cudaMemsetAsync(L->dcnt.p, 0, sizeof(DevCounts), L->stream))) return cuda_err(P, e, "graph counts");
    L->gm = true;
    st = solve_entry(L, G->src[i], G->q[i], G->N[i], G->tgt[i], G->M[i], G->psi[i], G->alpha[i]);
    if (st != SFMM_OK) {
        L->gm = false;
        return plan_error(P, st, "shell " + std::to_string(i) + " (graph mode): " + L->err);
    }
    DevCounts h;
    if ((e = cudaMemcpyAsync(&h, L->dcnt.p, sizeof h, cudaMemcpyDeviceToHost, L->stream)) ||
        (e = cudaStreamSynchronize(L->stream)))
        return cuda_err(P, e, "graph-mode solve");
    if (h.overflow) {
        L->gm = false;
        return plan_error(P, SFMM_ECUDA, "shell " + std::to_string(i) +
                                             ": the graph-mode solve overflowed the capacities planned from it");
    }
    return SFMM_OK;
}

void drop_graph(GraphState* G)
{
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    G->exec = nullptr;
    G->graph = nullptr;
}

// Record every shell's graph-mode solve (and the copy of its counts to the
// pinned reports) into one graph and instantiate it.
sfmm_status record(sfmm_plan_s* P, GraphState* G)
{
    drop_graph(G);
    cudaError_t e;
    const int64_t before = launch_total();
    if ((e = cudaStreamBeginCapture(G->origin, cudaStreamCaptureModeRelaxed))) return cuda_err(P, e, "begin capture");
    sfmm_status st = SFMM_OK;
    std::string where;
    e = cudaEventRecord(G->ev_fork, G->origin);
    for (int i = 0; i < G->n && !e && st == SFMM_OK; ++i) {
        sfmm_plan_s* L = G->shells[i];
        if ((e = cudaStreamWaitEvent(L->stream, G->ev_fork, 0))) break;
        st = solve_entry(L, G->src[i], G->q[i], G->N[i], G->tgt[i], G->M[i], G->psi[i], G->alpha[i]);
        if (st != SFMM_OK) {
            where = "shell " + std::to_string(i) + ": " + L->err;
            break;
        }
        if ((e = cudaMemcpyAsync(&G->h_rep[i].dc, L->dcnt.p, sizeof(DevCounts), cudaMemcpyDeviceToHost, L->stream)))
            break;
        // the walk's pair counts: graph mode leaves them in the plan's counter words
        if (L->d_m2l && (e = cudaMemcpyAsync(&G->h_rep[i].n_m2l, L->d_m2l, 8, cudaMemcpyDeviceToHost, L->stream))) break;
        if (L->d_p2p && (e = cudaMemcpyAsync(&G->h_rep[i].n_p2p, L->d_p2p, 8, cudaMemcpyDeviceToHost, L->stream))) break;
        if ((e = cudaEventRecord(G->ev_done[i], L->stream)) || (e = cudaStreamWaitEvent(G->origin, G->ev_done[i], 0)))
            break;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(G->origin, &g);
    count_launch(-(int)(launch_total() - before));     // recorded, not launched
    if (st != SFMM_OK) {
        if (g) cudaGraphDestroy(g);
        return plan_error(P, st, "graph recording, " + where);
    }
    if (e || e_end) {
        if (g) cudaGraphDestroy(g);
        return cuda_err(P, e ? e : e_end, "graph recording");
    }
    G->graph = g;
    size_t n_nodes = 0;
    if ((e = cudaGraphGetNodes(g, nullptr, &n_nodes))) return cuda_err(P, e, "graph nodes");
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes && (e = cudaGraphGetNodes(g, nodes.data(), &n_nodes))) return cuda_err(P, e, "graph nodes");
    G->kernel_nodes = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++G->kernel_nodes;
    }
    if ((e = cudaGraphInstantiate(&G->exec, g, 0))) {
        G->exec = nullptr;
        return cuda_err(P, e, "graph instantiation");
    }
    return SFMM_OK;
}

}  // namespace

void graph_release(sfmm_plan_s* P)
{
    GraphState* G = P->graph;
    if (!G) return;
    if (G->origin) cudaStreamSynchronize(G->origin);
    drop_graph(G);
    for (sfmm_plan_s* L : G->shells) sfmm_destroy(L);
    for (cudaEvent_t ev : G->ev_done)
        if (ev) cudaEventDestroy(ev);
    if (G->ev_fork) cudaEventDestroy(G->ev_fork);
    if (G->origin) cudaStreamDestroy(G->origin);
    if (G->h_rep) cudaFreeHost(G->h_rep);
    delete G;
    P->graph = nullptr;
}

}  // namespace sfmm

using namespace sfmm;

extern "C" {

sfmm_status sfmm_graph_capture(sfmm_plan_t plan, int n_shells, const double* const* src_xyz, const void* const* q,
                               const int64_t* N, const double* const* tgt_xyz, const int64_t* M, double* const* psi,
                               double* const* alpha, double slack)
{
    if (!plan) return SFMM_EINVAL;
    graph_release(plan);
    if (n_shells < 1) return plan_error(plan, SFMM_EINVAL, "n_shells must be >= 1");
    if (!src_xyz || !q || !N || !tgt_xyz || !M || !alpha)
        return plan_error(plan, SFMM_EINVAL, "NULL array of shells");
    if (!(slack >= 0.0 && slack <= 16.0)) return plan_error(plan, SFMM_EINVAL, "slack must be in [0, 16]");
    if (plan->opt.precision == SFMM_FP32)
        return plan_error(plan, SFMM_EINVAL, "graph-launched shells run SFMM_FP64, SFMM_MIXED or SFMM_MIXED_DF plans");
    if (plan->opt.sigma > 0.0)
        return plan_error(plan, SFMM_EINVAL, "graph-launched shells run point masses only (sigma == 0)");
    for (int i = 0; i < n_shells; ++i) {
        if (N[i] < 0 || M[i] < 0 || N[i] > 0x7fffffffLL || M[i] > 0x7fffffffLL)
            return plan_error(plan, SFMM_EINVAL, "N and M must be in [0, 2^31)");
        if ((N[i] > 0 && (!src_xyz[i] || !q[i])) || (M[i] > 0 && (!tgt_xyz[i] || !alpha[i])))
            return plan_error(plan, SFMM_EINVAL, "NULL array of shell " + std::to_string(i));
    }
    auto* G = new (std::nothrow) GraphState();
    if (!G) return SFMM_ENOMEM;
    plan->graph = G;
    G->n = n_shells;
    G->slack = slack > 0.0 ? slack : 0.25;
    G->src.assign(src_xyz, src_xyz + n_shells);
    G->q.assign(q, q + n_shells);
    G->N.assign(N, N + n_shells);
    G->tgt.assign(tgt_xyz, tgt_xyz + n_shells);
    G->M.assign(M, M + n_shells);
    G->alpha.assign(alpha, alpha + n_shells);
    G->psi.assign(n_shells, nullptr);
    if (psi) G->psi.assign(psi, psi + n_shells);
    G->ev_done.assign(n_shells, nullptr);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&G->origin, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&G->ev_fork, cudaEventDisableTiming)) ||
        (e = cudaMallocHost(&G->h_rep, sizeof(ShellReport) * (size_t)n_shells))) {
        graph_release(plan);
        return cuda_err(plan, e, "graph setup");
    }
    memset(G->h_rep, 0, sizeof(ShellReport) * (size_t)n_shells);
    for (int i = 0; i < n_shells; ++i)
        if ((e = cudaEventCreateWithFlags(&G->ev_done[i], cudaEventDisableTiming))) {
            graph_release(plan);
            return cuda_err(plan, e, "graph setup");
        }
    // the shells start after the work already queued on the plan's stream
    if ((e = cudaStreamSynchronize(plan->stream))) {
        graph_release(plan);
        return cuda_err(plan, e, "graph setup");
    }
    for (int i = 0; i < n_shells; ++i) {
        sfmm_options o = plan->opt;
        cudaStream_t st = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) {
            graph_release(plan);
            return cuda_err(plan, e, "shell stream");
        }
        o.stream = st;
        o.n_max = o.m_max = 0;
        sfmm_plan_t L = nullptr;
        sfmm_status ps = sfmm_plan(&L, plan->max_depth, plan->p, plan->tol, &o);
        if (ps != SFMM_OK) {
            cudaStreamDestroy(st);
            graph_release(plan);
            return plan_error(plan, ps, "could not create a shell solver");
        }
        L->owns_stream = true;
        G->shells.push_back(L);
        if ((ps = prepare_shell(plan, G, i)) != SFMM_OK) {
            const std::string msg = plan->err;
            graph_release(plan);
            return plan_error(plan, ps, msg);
        }
    }
    sfmm_status st = record(plan, G);
    if (st != SFMM_OK) {
        const std::string msg = plan->err;
        graph_release(plan);
        return plan_error(plan, st, msg);
    }
    return SFMM_OK;
}

sfmm_status sfmm_graph_launch(sfmm_plan_t plan)
{
    if (!plan) return SFMM_EINVAL;
    GraphState* G = plan->graph;
    if (!G || !G->exec) return plan_error(plan, SFMM_EINVAL, "no graph: call sfmm_graph_capture first");
    cudaError_t e;
    if ((e = cudaGraphLaunch(G->exec, plan->stream))) return cuda_err(plan, e, "graph launch");
    count_launch((int)G->kernel_nodes);
    if ((e = cudaStreamSynchronize(plan->stream))) return cuda_err(plan, e, "graph replay");
    ++G->launches;
    bool again = false;
    for (int i = 0; i < G->n; ++i) {
        if (!G->h_rep[i].dc.overflow) continue;
        // this shell outgrew a capacity: solve it synchronously (its results
        // replace the replay's), plan its capacities anew and record again
        ++G->overflows;
        sfmm_status st = prepare_shell(plan, G, i);
        if (st != SFMM_OK) return st;
        again = true;
    }
    if (again) {
        ++G->recaptures;
        sfmm_status st = record(plan, G);
        if (st != SFMM_OK) return st;
    }
    return SFMM_OK;
}

sfmm_status sfmm_graph_info(sfmm_plan_t plan, sfmm_graph_stats* out)
{
    if (!plan || !out) return SFMM_EINVAL;
    memset(out, 0, sizeof *out);
    GraphState* G = plan->graph;
    if (!G) return SFMM_OK;
    out->n_shells = G->n;
    out->kernel_nodes = G->kernel_nodes;
    out->launches = G->launches;
    out->overflows = G->overflows;
    out->recaptures = G->recaptures;
    for (int i = 0; i < G->n; ++i) {
        const ShellReport& r = G->h_rep[i];
        out->n_nodes += r.dc.nn;
        out->n_leaves += r.dc.n_leaves;
        out->n_m2l += r.n_m2l;
        out->n_p2p += r.n_p2p;
    }
    return SFMM_OK;
}

sfmm_status sfmm_graph_release(sfmm_plan_t plan)
{
    if (!plan) return SFMM_EINVAL;
    graph_release(plan);
    return SFMM_OK;
}

}  // extern "C"
