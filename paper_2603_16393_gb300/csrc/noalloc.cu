// noalloc.cu -- fwi_w2_misfit_static: the W2 misfit entry point without a
// caller-provided workspace.
//
// fwi_w2_misfit needs a little device scratch (one float per trace, the
// per-trace W2 values that are summed into J) that normally lives in the
// caller's workspace.  Some callers cannot hand out device memory: code that
// runs inside a host framework which owns every device allocation through its
// own pool and forbids side allocations, or a steady-state loop in which an
// allocation (and the device synchronisation it may imply) is not allowed.
// This entry point uses a scratch array compiled into the library instead.
//
// The array lives in device global memory of every GPU that loads the
// library, for as long as the process runs.  Its device address is looked up
// (cudaGetSymbolAddress) the first time the entry point is called on a
// device, with that device current; make that first call before any stream
// capture begins.  The address belongs to the device's current context: a
// cudaDeviceReset (or any other end of that context) reloads the module at a
// new address, so the lookup is repeated on the first call in a new context.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

// per-trace W2 scratch shared by every call on a device
static __device__ __align__(256) float g_w2_scratch[FWI_STATIC_MAX_TRACES];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
    float *ptr = nullptr;
    unsigned long long ctx_id = 0;   // context the address belongs to
    bool ctx_known = false;
};
ScratchSlot g_slot[kMaxDevices];
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (the driver entry points
// are fetched through the runtime, so the library needs no link to the
// driver library).  Returns false when the driver cannot tell.
bool current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_w2_scratch in the current device's current context
// (looked up once per device and context).  Returns nullptr and the CUDA
// error on failure.
float *scratch_on_current_device(cudaError_t *err)
{
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    unsigned long long id = 0;
    bool known = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchSlot &sl = g_slot[dev];
    if (!sl.ptr || !known || !sl.ctx_known || sl.ctx_id != id) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_w2_scratch);
        if (*err != cudaSuccess) return nullptr;
        // the lookup makes the primary context current if it was not yet
        known = current_context_id(&id);
        sl.ptr = static_cast<float *>(p);
        sl.ctx_id = id;
        sl.ctx_known = known;
    }
    *err = cudaSuccess;
    return sl.ptr;
}

}  // namespace

}  // namespace fwi

extern "C" FWI_API fwi_status fwi_w2_misfit_static(const fwi_plan *plan, const void *obs_ctx,
                                                   const float *d_syn, float *J, float *w2,
                                                   float *adj_src, void *stream)
{
    if (!plan || !obs_ctx || !d_syn || !J)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "plan, obs_ctx, d_syn and J must not be NULL");
    const fwi::Plan &pl = *reinterpret_cast<const fwi::Plan *>(plan);
    cudaError_t e = cudaSuccess;
    float *scratch = nullptr;
    if (!w2) {
        // the per-trace values go to the built-in array only when the caller
        // does not take them
        const long long ntraces = (long long)pl.p.batch * pl.p.ns * pl.p.nr;
        if (ntraces > FWI_STATIC_MAX_TRACES)
            return fwi::record_error(FWI_ERR_UNSUPPORTED,
                                     "fwi_w2_misfit_static: %lld traces (batch x ns x nr) exceed "
                                     "its built-in scratch of %d traces; pass w2 or use "
                                     "fwi_w2_misfit",
                                     ntraces, FWI_STATIC_MAX_TRACES);
        scratch = fwi::scratch_on_current_device(&e);
        if (!scratch)
            return fwi::record_error(FWI_ERR_CUDA, "fwi_w2_misfit_static scratch lookup: %s",
                                     cudaGetErrorString(e));
    }
    e = fwi::launch_w2_misfit(pl, (const unsigned char *)obs_ctx, d_syn, J, w2, adj_src, scratch,
                              (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_w2_misfit_static launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}
