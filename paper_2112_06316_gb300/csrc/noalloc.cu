// ifgf_apply_noalloc: the operator apply with its workspace in a fixed,
// file-scope device array instead of memory obtained from cudaMalloc.
//
// The workspace of an apply (w*sigma and the accumulated field in Morton order,
// plus the cone values F of every level) normally lives in plan-owned device
// memory that ifgf_apply grows with cudaMalloc the first time a larger nrhs or
// another precision is requested.  This entry point places the same workspace in
// g_scratch below, so the call itself allocates and frees nothing.
#include <mutex>

#include "ifgf_internal.h"

namespace ifgf {

// Largest workspace the allocation-free apply accepts (bytes).
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

// Shared by every call on a device; it keeps whatever the last call wrote.
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

ifgf_status run_apply_on(Plan &p, const Workspace &ws, const void *sigma, void *y, int nrhs, int prec,
                         cudaStream_t s);
ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
void clear_error();

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};  // id of the context the cached address belongs to

// Driver calls that identify the calling thread's current context, resolved through the runtime
// (no link-time dependency on the driver library).  Context ids are unique for the life of the
// process, so a context created after cudaDeviceReset never matches an earlier one.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

bool current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (CtxGetCurrentFn)f1;
            get_id = (CtxGetIdFn)f2;
        }
        resolved = true;
    }
    void *ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of g_scratch on the current device, looked up once per device and context.
// In host code the name g_scratch is only a host-side stand-in for the symbol, not a device
// address, so kernels must receive the address returned here.  The lookup is repeated only when
// the device's context has changed (after cudaDeviceReset the module is loaded again and the
// array may sit elsewhere); where the context cannot be identified the first address is kept.
ifgf_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return IFGF_EUNSUPPORTED;
    }
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev] || (have_ctx && g_ctx[dev] != ctx)) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
            return IFGF_ECUDA;
        }
        g_addr[dev] = ptr;
        g_ctx[dev] = have_ctx ? ctx : 0;
    }
    *out = g_addr[dev];
    return IFGF_OK;
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_apply_noalloc(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs,
                                          ifgf_precision prec, void *stream) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || (nrhs > 0 && (!sigma_dev || !y_dev))) {
        set_error("invalid nrhs or null device pointer");
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    if (nrhs == 0) return IFGF_OK;
    if (sigma_dev == y_dev) {
        set_error("sigma and y must not alias");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    // same layout as the plan-owned workspace
    WorkspaceLayout lay;
    const size_t total = workspace_layout(p, nrhs, (int)prec, lay);
    if (total > kNoAllocScratchBytes) {
        set_error("ifgf_apply_noalloc: workspace of %zu bytes exceeds the fixed %zu-byte scratch (N=%lld, nrhs=%d); "
                  "use ifgf_apply", total, kNoAllocScratchBytes, (long long)p.N, nrhs);
        return IFGF_EINVAL;
    }
    void *base = nullptr;
    ifgf_status st = scratch_address(&base);
    if (st != IFGF_OK) return st;
    Workspace ws;
    workspace_bind(ws, p, base, lay, nrhs, (int)prec);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_apply_on(p, ws, sigma_dev, y_dev, nrhs, (int)prec, s);
    if (st != IFGF_OK) return st;
    return apply_correction(p, sigma_dev, y_dev, nrhs, (int)prec, s);
}
