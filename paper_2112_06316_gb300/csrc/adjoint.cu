// Host side of the adjoint apply A^H g (conjugate transpose of the discrete
// operator, including the correction) and of the vector-Jacobian product
// (A^H g, Re <g, dA/dk sigma>): builds the anterpolation lists on the first call,
// manages the adjoint workspace and dispatches over the compiled interpolation
// orders (kernels in fwd_kernels.cuh).
#include <cmath>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {

template <int PS, int PA>
ifgf_status run_adjoint_t(Plan &p, const void *g, void *out, int nrhs, int prec, cudaStream_t s, void *gs, void *bws,
                          void **G, void *const *Fd, double *dk_partials);
template <int PS, int PA>
ifgf_status run_dk_t(Plan &p, int nrhs, int prec, cudaStream_t s, const void *gs, void **G, double *partials,
                     long long *nparts);
#define IFGF_EXTERN(a, b)                                                                                           \
    extern template ifgf_status run_adjoint_t<a, b>(Plan &, const void *, void *, int, int, cudaStream_t, void *,     \
                                                    void *, void **, void *const *, double *);                      \
    extern template ifgf_status run_dk_t<a, b>(Plan &, int, int, cudaStream_t, const void *, void **, double *,       \
                                               long long *);
IFGF_EXTERN(3, 5)
IFGF_EXTERN(4, 6)
IFGF_EXTERN(5, 7)
IFGF_EXTERN(5, 8)
IFGF_EXTERN(6, 8)
#undef IFGF_EXTERN

ifgf_status apply_correction_adjoint(Plan &p, const void *g, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status run_apply_on(Plan &p, const Workspace &ws, const void *sigma, void *y, int nrhs, int prec,
                         cudaStream_t s);
void clear_error();

namespace {

ifgf_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
}

// Anterpolation lists per level (host build, then upload); once per plan.
ifgf_status ensure_adjoint_lists(Plan &p, cudaStream_t s) {
    if (p.adj_ready) return IFGF_OK;
    int64_t maxe = p.N;
    for (int d = 3; d < p.D; d++) maxe = std::max<int64_t>(maxe, p.N + p.lv[d].nrc * p.P);
    if (maxe >= (int64_t)0x7fffffff) {
        set_error("adjoint lists exceed the 32-bit entry range");
        return IFGF_EUNSUPPORTED;
    }
    ifgf_status st = build_adjoint_lists(p, p.xs.data());
    if (st != IFGF_OK) return st;
    for (int d = 3; d <= p.D; d++) {
        HostLevel &L = p.lv[d];
        void *a = nullptr, *b = nullptr;
        cudaError_t e = cudaMalloc(&a, sizeof(int64_t) * L.ad_start.size());
        if (e == cudaSuccess) e = cudaMalloc(&b, sizeof(int) * (L.ad_list.size() + 1));
        if (e != cudaSuccess) {
            if (a) cudaFree(a);
            return cuda_fail(e, "adjoint list allocation");
        }
        p.allocs.push_back(a);
        p.allocs.push_back(b);
        p.device_bytes += (int64_t)(sizeof(int64_t) * L.ad_start.size() + sizeof(int) * (L.ad_list.size() + 1));
        e = cudaMemcpyAsync(a, L.ad_start.data(), sizeof(int64_t) * L.ad_start.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !L.ad_list.empty())
            e = cudaMemcpyAsync(b, L.ad_list.data(), sizeof(int) * L.ad_list.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint list upload");
        p.d_ad_start[d] = (int64_t *)a;
        p.d_ad_list[d] = (int *)b;
        std::vector<int64_t>().swap(L.ad_start);
        std::vector<int>().swap(L.ad_list);
    }
    p.adj_ready = true;
    return IFGF_OK;
}

// A^H g into out (without the correction); leaves the gathered g and the cone
// values G of every level in the adjoint workspace (returned through gs_out / G).
// With Fd (the forward cone values of every level) the anterpolation also writes the
// cousin and propagation parts of Re <g, dA/dk sigma>, one double per relevant cone
// and level in order, to dk_partials.
ifgf_status adjoint_core(Plan &p, const void *g_dev, void *out_dev, int nrhs, int prec, cudaStream_t s, void **gs_out,
                         void **G, void *const *Fd = nullptr, double *dk_partials = nullptr) {
    ifgf_status st = ensure_adjoint_lists(p, s);
    if (st != IFGF_OK) return st;
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0, oG[IFGF_MAXD + 1] = {};
    const size_t ogs = off;
    off += al(cb * p.N * nrhs);
    const size_t ob = off;
    off += al(cb * p.N * nrhs);
    for (int d = 3; d <= p.D; d++) {
        oG[d] = off;
        off += al(cb * (size_t)nrhs * p.lv[d].nrc * p.lv[d].nfac * p.Pstride);
    }
    if (off > p.adj_ws_bytes) {
        if (p.adj_ws) cudaFree(p.adj_ws);
        p.adj_ws = nullptr;
        p.adj_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&p.adj_ws, off);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint workspace");
        p.adj_ws_bytes = off;
    }
    char *c = (char *)p.adj_ws;
    for (int d = 3; d <= p.D; d++) G[d] = c + oG[d];
    *gs_out = c + ogs;
#define IFGF_CASE(a, b)                                                                                     \
    if (p.Ps == a && p.Pang == b)                                                                           \
        return run_adjoint_t<a, b>(p, g_dev, out_dev, nrhs, prec, s, c + ogs, c + ob, G, Fd, dk_partials);
    IFGF_CASE(3, 5)
    IFGF_CASE(4, 6)
    IFGF_CASE(5, 7)
    IFGF_CASE(5, 8)
    IFGF_CASE(6, 8)
#undef IFGF_CASE
    set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    return IFGF_EUNSUPPORTED;
}

ifgf_status run_dk(Plan &p, int nrhs, int prec, cudaStream_t s, const void *gs, void **G, double *partials,
                   long long *nparts) {
#define IFGF_CASE(a, b) \
    if (p.Ps == a && p.Pang == b) return run_dk_t<a, b>(p, nrhs, prec, s, gs, G, partials, nparts);
    IFGF_CASE(3, 5)
    IFGF_CASE(4, 6)
    IFGF_CASE(5, 7)
    IFGF_CASE(5, 8)
    IFGF_CASE(6, 8)
#undef IFGF_CASE
    set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    return IFGF_EUNSUPPORTED;
}

ifgf_status check_args(ifgf_plan *plan, const void *a, void *b, int nrhs, ifgf_precision prec) {
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || (nrhs > 0 && (!a || !b))) {
        set_error("invalid nrhs or null device pointer");
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    if (nrhs > 0 && a == b) {
        set_error("input and output must not alias");
        return IFGF_EINVAL;
    }
    return IFGF_OK;
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_apply_adjoint(ifgf_plan *plan, const void *g_dev, void *out_dev, int nrhs,
                                          ifgf_precision prec, void *stream) {
    clear_error();
    ifgf_status st = check_args(plan, g_dev, out_dev, nrhs, prec);
    if (st != IFGF_OK || nrhs == 0) return st;
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    void *gs = nullptr, *G[IFGF_MAXD + 1] = {};
    st = adjoint_core(p, g_dev, out_dev, nrhs, (int)prec, s, &gs, G);
    if (st != IFGF_OK) return st;
    return apply_correction_adjoint(p, g_dev, out_dev, nrhs, (int)prec, s);
}

namespace ifgf {
namespace {

// Gradient part of the vector-Jacobian product on a forward state `fwd` (w sigma and the cone
// values of every level left by a forward apply of sigma): gsigma = A^H g and, when dk_host is
// given, dk = Re <g, dA/dk sigma> (near field and leaf evaluation by their own reductions, the
// cousin and propagation terms inside the fused anterpolation).
ifgf_status vjp_core(Plan &p, const Workspace &fwd, const void *g_dev, void *gsigma_dev, int nrhs, double *dk_host,
                     int prec, cudaStream_t s) {
    double *partials = nullptr;
    long long need = 0;
    if (dk_host) {
        // per relevant cone (fused anterpolation), then the near field and the leaf: FP64 by their own
        // passes (one block per 128 targets / nodes), mixed inside the adjoint kernels (one block per
        // 128 sources / per four leaf chunks)
        need = (p.N + 127) / 128 + std::max<long long>((p.lv[p.D].nrc * p.P + 127) / 128, (p.ncchunk[p.D] + 3) / 4);
        for (int d = 3; d <= p.D; d++) need += p.lv[d].nrc;
        for (int d = 3; d < p.D; d++)  // adaptive tree: the leaves of the coarser levels (per 128 sources / nodes)
            if (p.nleaf_rc[d]) need += std::max<long long>((p.N + 127) / 128, ((long long)p.nleaf_rc[d] * p.P + 127) / 128);
        const size_t bytes = sizeof(double) * (need + 1);
        if (bytes > p.dk_ws_bytes) {
            if (p.dk_ws) cudaFree(p.dk_ws);
            p.dk_ws = nullptr;
            p.dk_ws_bytes = 0;
            cudaError_t e = cudaMalloc(&p.dk_ws, bytes);
            if (e != cudaSuccess) return cuda_fail(e, "k-gradient workspace");
            p.dk_ws_bytes = bytes;
        }
        partials = (double *)p.dk_ws;
    }
    void *gs = nullptr, *G[IFGF_MAXD + 1] = {};
    void *Fd[IFGF_MAXD + 1] = {};
    for (int d = 3; d <= p.D; d++) Fd[d] = fwd.F[d];
    const Workspace saved = p.ws;
    p.ws = fwd;  // the k-derivative reads w sigma and the cone values of the forward state
    ifgf_status st = adjoint_core(p, g_dev, gsigma_dev, nrhs, prec, s, &gs, G, dk_host ? Fd : nullptr, partials);
    p.ws = saved;
    if (st != IFGF_OK) return st;
    st = apply_correction_adjoint(p, g_dev, gsigma_dev, nrhs, prec, s);
    if (st != IFGF_OK || !dk_host) return st;
    long long np = 0;
    for (int d = 3; d <= p.D; d++) np += p.lv[d].nrc;
    if (prec == IFGF_MIXED) {  // near field and leaf reduced inside the adjoint kernels
        np += (p.N + 127) / 128;
        if (p.lv[p.D].nrc) np += (p.ncchunk[p.D] + 3) / 4;
        for (int d = 3; d < p.D; d++)
            if (p.nleaf_rc[d]) np += (p.N + 127) / 128;
    } else {
        long long nd = 0;
        p.ws = fwd;
        st = run_dk(p, nrhs, prec, s, gs, G, partials + np, &nd);
        p.ws = saved;
        if (st != IFGF_OK) return st;
        np += nd;
    }
    std::vector<double> h(np > 0 ? np : 1, 0.0);
    if (np > 0) {
        cudaError_t e = cudaMemcpyAsync(h.data(), partials, sizeof(double) * np, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "vjp partial copy");
    }
    double sum = 0.0;
    for (long long i = 0; i < np; i++) sum += h[i];
    *dk_host = sum;
    return IFGF_OK;
}

// Caller-provided workspace: checks its size and alignment and lays the parts out in it.
ifgf_status bind_user_workspace(const Plan &p, void *ws_dev, int64_t ws_bytes, int nrhs, int prec, Workspace &ws) {
    WorkspaceLayout lay;
    const size_t need = workspace_layout(p, nrhs, prec, lay);
    if (!ws_dev || ws_bytes < 0 || (size_t)ws_bytes < need || ((uintptr_t)ws_dev & 255) != 0) {
        set_error("workspace must be a 256-byte aligned device buffer of at least %zu bytes (got %lld at %p)", need,
                  (long long)ws_bytes, ws_dev);
        return IFGF_EINVAL;
    }
    workspace_bind(ws, p, ws_dev, lay, nrhs, prec);
    return IFGF_OK;
}

}  // namespace
}  // namespace ifgf

extern "C" ifgf_status ifgf_apply_vjp(ifgf_plan *plan, const void *sigma_dev, const void *g_dev, void *gsigma_dev,
                                      int nrhs, double *dk_host, ifgf_precision prec, void *stream) {
    clear_error();
    ifgf_status st = check_args(plan, g_dev, gsigma_dev, nrhs, prec);
    if (st != IFGF_OK) return st;
    if (nrhs > 0 && (!sigma_dev || sigma_dev == gsigma_dev || sigma_dev == g_dev)) {
        set_error("sigma must be a distinct, non-null device buffer");
        return IFGF_EINVAL;
    }
    if (dk_host) *dk_host = 0.0;
    if (nrhs == 0) return IFGF_OK;
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    // forward state (a = w sigma, cone values F) in the plan workspace; gsigma is scratch here
    st = run_apply(p, sigma_dev, gsigma_dev, nrhs, (int)prec, s);
    if (st != IFGF_OK) return st;
    return vjp_core(p, p.ws, g_dev, gsigma_dev, nrhs, dk_host, (int)prec, s);
}

extern "C" ifgf_status ifgf_plan_workspace_bytes(const ifgf_plan *plan, int nrhs, ifgf_precision prec,
                                                 int64_t *bytes) {
    clear_error();
    if (!plan || !bytes || nrhs < 0 || (prec != IFGF_FP64 && prec != IFGF_MIXED)) {
        set_error("null plan or output, negative nrhs or unknown precision");
        return IFGF_EINVAL;
    }
    WorkspaceLayout lay;
    *bytes = (int64_t)workspace_layout(plan->p, nrhs, (int)prec, lay);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_apply_ws(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs,
                                     ifgf_precision prec, void *ws_dev, int64_t ws_bytes, void *stream) {
    clear_error();
    ifgf_status st = check_args(plan, sigma_dev, y_dev, nrhs, prec);
    if (st != IFGF_OK || nrhs == 0) return st;
    Plan &p = plan->p;
    Workspace ws;
    st = bind_user_workspace(p, ws_dev, ws_bytes, nrhs, (int)prec, ws);
    if (st != IFGF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = run_apply_on(p, ws, sigma_dev, y_dev, nrhs, (int)prec, s);
    if (st != IFGF_OK) return st;
    return apply_correction(p, sigma_dev, y_dev, nrhs, (int)prec, s);
}

extern "C" ifgf_status ifgf_apply_vjp_ws(ifgf_plan *plan, const void *ws_dev, int64_t ws_bytes, const void *g_dev,
                                         void *gsigma_dev, int nrhs, double *dk_host, ifgf_precision prec,
                                         void *stream) {
    clear_error();
    ifgf_status st = check_args(plan, g_dev, gsigma_dev, nrhs, prec);
    if (st != IFGF_OK) return st;
    if (dk_host) *dk_host = 0.0;
    if (nrhs == 0) return IFGF_OK;
    Plan &p = plan->p;
    Workspace ws;
    st = bind_user_workspace(p, const_cast<void *>(ws_dev), ws_bytes, nrhs, (int)prec, ws);
    if (st != IFGF_OK) return st;
    if ((const void *)gsigma_dev == ws_dev || g_dev == ws_dev) {
        set_error("the workspace must not alias g or gsigma");
        return IFGF_EINVAL;
    }
    return vjp_core(p, ws, g_dev, gsigma_dev, nrhs, dk_host, (int)prec, (cudaStream_t)stream);
}
