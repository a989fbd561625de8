// Batched apply over several plans (many scatterers, many right-hand sides) as
// one CUDA graph.  The launch sequences of all plans are captured once on a
// private stream, forked over `nstreams` capture streams so independent
// scatterers overlap on the GPU, and joined; later calls with the same buffers
// replay the instantiated graph with a single cudaGraphLaunch.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {
ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status ensure_workspace(Plan &p, int nrhs, int prec);
ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
void clear_error();
}  // namespace ifgf

using namespace ifgf;

struct ifgf_group {
    std::vector<ifgf_plan *> plans;
    int nstreams = 4;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // buffers and sizes the graph was captured with
    std::vector<const void *> cap_sigma;
    std::vector<void *> cap_y;
    std::vector<int> cap_nrhs;
    std::vector<uint64_t> cap_gen;
    int cap_prec = -1;
    int cap_nstreams = -1;
    int device = -1;
    int64_t captures = 0;  // graphs captured so far
};

static void drop_graph(ifgf_group *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
    g->cap_sigma.clear();
}

static ifgf_status gfail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
}

extern "C" {

ifgf_status ifgf_group_create(ifgf_plan *const *plans, int nplans, ifgf_group **out) {
    clear_error();
    if (out) *out = nullptr;
    if (!out || nplans < 1 || !plans) {
        set_error("invalid group arguments");
        return IFGF_EINVAL;
    }
    for (int i = 0; i < nplans; i++) {
        if (!plans[i]) {
            set_error("null plan %d in group", i);
            return IFGF_EINVAL;
        }
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) {
                set_error("plan %d appears twice in the group (its workspace would be shared)", i);
                return IFGF_EINVAL;
            }
    }
    ifgf_group *g = new ifgf_group();
    g->plans.assign(plans, plans + nplans);
    cudaGetDevice(&g->device);
    *out = g;
    return IFGF_OK;
}

ifgf_status ifgf_group_set_streams(ifgf_group *g, int nstreams) {
    clear_error();
    if (!g || nstreams < 1 || nstreams > 64) {
        set_error("nstreams must be in 1..64");
        return IFGF_EINVAL;
    }
    if (nstreams != g->nstreams) drop_graph(g);
    g->nstreams = nstreams;
    return IFGF_OK;
}

ifgf_status ifgf_group_captures(const ifgf_group *g, int64_t *captures) {
    clear_error();
    if (!g || !captures) {
        set_error("null group or output");
        return IFGF_EINVAL;
    }
    *captures = g->captures;
    return IFGF_OK;
}

void ifgf_group_destroy(ifgf_group *g) {
    if (!g) return;
    drop_graph(g);
    for (cudaStream_t s : g->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    delete g;
}

ifgf_status ifgf_group_apply(ifgf_group *g, const void *const *sigma, void *const *y, const int *nrhs,
                             ifgf_precision prec, void *stream) {
    clear_error();
    if (!g || !sigma || !y || !nrhs) {
        set_error("invalid group apply arguments");
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    const int n = (int)g->plans.size();
    for (int i = 0; i < n; i++) {
        if (nrhs[i] < 0 || (nrhs[i] > 0 && (!sigma[i] || !y[i] || sigma[i] == y[i]))) {
            set_error("invalid buffers or nrhs for plan %d", i);
            return IFGF_EINVAL;
        }
    }
    const cudaStream_t cs = (cudaStream_t)stream;
    bool same = g->exec && g->cap_prec == (int)prec && g->cap_nstreams == g->nstreams;
    for (int i = 0; same && i < n; i++)
        same = g->cap_sigma[i] == sigma[i] && g->cap_y[i] == y[i] && g->cap_nrhs[i] == nrhs[i] &&
               g->cap_gen[i] == g->plans[i]->p.gen;
    if (!same) {
        drop_graph(g);
        // every workspace must exist before capture (no allocation inside a capture)
        for (int i = 0; i < n; i++) {
            if (nrhs[i] == 0) continue;
            Plan &p = g->plans[i]->p;
            p.profile = false;
            ifgf_status st = ensure_workspace(p, nrhs[i], (int)prec);
            if (st != IFGF_OK) return st;
        }
        const int S = g->nstreams;
        while ((int)g->streams.size() < S + 1) {
            cudaStream_t s;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) return gfail(e, "cudaStreamCreate");
            g->streams.push_back(s);
        }
        while ((int)g->events.size() < S + 1) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return gfail(e, "cudaEventCreate");
            g->events.push_back(ev);
        }
        cudaStream_t s0 = g->streams[0];
        cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return gfail(e, "cudaStreamBeginCapture");
        ifgf_status st = IFGF_OK;
        cudaEventRecord(g->events[0], s0);
        for (int k = 1; k <= S; k++) cudaStreamWaitEvent(g->streams[k], g->events[0], 0);
        // largest plans first, assigned round-robin to the capture streams
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (int64_t)g->plans[a]->p.N * nrhs[a] > (int64_t)g->plans[b]->p.N * nrhs[b];
        });
        for (int t = 0; t < n && st == IFGF_OK; t++) {
            const int i = order[t];
            if (nrhs[i] == 0) continue;
            cudaStream_t si = g->streams[1 + t % S];
            Plan &p = g->plans[i]->p;
            st = run_apply(p, sigma[i], y[i], nrhs[i], (int)prec, si);
            if (st == IFGF_OK) st = apply_correction(p, sigma[i], y[i], nrhs[i], (int)prec, si);
        }
        for (int k = 1; k <= S; k++) {
            cudaEventRecord(g->events[k], g->streams[k]);
            cudaStreamWaitEvent(s0, g->events[k], 0);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s0, &graph);
        if (st != IFGF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return gfail(e, "cudaStreamEndCapture");
        g->graph = graph;
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) {
            drop_graph(g);
            return gfail(e, "cudaGraphInstantiate");
        }
        g->cap_sigma.assign(sigma, sigma + n);
        g->cap_y.assign(y, y + n);
        g->cap_nrhs.assign(nrhs, nrhs + n);
        g->cap_gen.resize(n);
        for (int i = 0; i < n; i++) g->cap_gen[i] = g->plans[i]->p.gen;
        g->cap_prec = (int)prec;
        g->cap_nstreams = g->nstreams;
        g->captures++;
    }
    cudaError_t e = cudaGraphLaunch(g->exec, cs);
    if (e != cudaSuccess) return gfail(e, "cudaGraphLaunch");
    return IFGF_OK;
}

}  // extern "C"
