// group.cu -- gradients of several plans (uneven grid sizes, any propagator
// families) as one unit: each plan's forward -> W2 misfit -> adjoint pipeline
// runs on a stream of its own, forked from the caller's stream by an event
// and joined back to it, so the plans' kernels overlap on the GPU and a
// capture of the caller's stream records the whole set as one CUDA graph.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "fwi_internal.cuh"

struct fwi_group {
    std::vector<const fwi_plan *> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
};

namespace {

void release(fwi_group *g)
{
    for (cudaStream_t s : g->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->joins)
        if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    delete g;
}

}  // namespace

extern "C" {

fwi_status fwi_group_create(const fwi_plan *const *plans, int n, fwi_group **out)
{
    if (!out) return fwi::record_error(FWI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || n < 1) return fwi::record_error(FWI_ERR_INVALID_ARG, "need n >= 1 plans");
    for (int i = 0; i < n; ++i)
        if (!plans[i]) return fwi::record_error(FWI_ERR_INVALID_ARG, "plan %d is NULL", i);
    fwi_group *g = new (std::nothrow) fwi_group();
    if (!g) return fwi::record_error(FWI_ERR_INVALID_ARG, "out of host memory");
    g->plans.assign(plans, plans + n);
    g->streams.assign(n, nullptr);
    g->joins.assign(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&g->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->joins[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release(g);
        return fwi::record_error(FWI_ERR_CUDA, "fwi_group_create: %s", cudaGetErrorString(e));
    }
    *out = g;
    return FWI_OK;
}

void fwi_group_destroy(fwi_group *g)
{
    if (g) release(g);
}

fwi_status fwi_group_gradient(fwi_group *g, const float *const *v, const void *const *obs_ctx,
                              float *const *d_syn, float *const *adj_src,
                              float *const *snapshots, float *const *grad, float *const *J,
                              void *const *workspace, void *stream)
{
    if (!g || !v || !obs_ctx || !d_syn || !adj_src || !snapshots || !grad || !J || !workspace)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "group and array lists must not be NULL");
    const int n = (int)g->plans.size();
    for (int i = 0; i < n; ++i)
        if (!v[i] || !obs_ctx[i] || !d_syn[i] || !adj_src[i] || !snapshots[i] || !grad[i] ||
            !J[i] || !workspace[i])
            return fwi::record_error(FWI_ERR_INVALID_ARG, "a buffer of plan %d is NULL", i);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(g->fork, st);
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_group_gradient: %s", cudaGetErrorString(e));
    fwi_status s = FWI_OK;
    int forked = 0;
    for (int i = 0; i < n && s == FWI_OK; ++i) {
        cudaStream_t si = g->streams[i];
        e = cudaStreamWaitEvent(si, g->fork, 0);
        if (e != cudaSuccess) {
            s = fwi::record_error(FWI_ERR_CUDA, "fwi_group_gradient: %s", cudaGetErrorString(e));
            break;
        }
        ++forked;
        s = fwi_forward(g->plans[i], v[i], d_syn[i], snapshots[i], workspace[i], si);
        if (s == FWI_OK)
            s = fwi_w2_misfit(g->plans[i], obs_ctx[i], d_syn[i], J[i], nullptr, adj_src[i],
                              workspace[i], si);
        if (s == FWI_OK)
            s = fwi_adjoint_grad(g->plans[i], v[i], adj_src[i], snapshots[i], grad[i],
                                 workspace[i], si);
    }
    // join every forked stream back (also after an error, so that a capture
    // of the caller's stream can end)
    for (int i = 0; i < forked; ++i) {
        cudaError_t ej = cudaEventRecord(g->joins[i], g->streams[i]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, g->joins[i], 0);
        if (ej != cudaSuccess && s == FWI_OK)
            s = fwi::record_error(FWI_ERR_CUDA, "fwi_group_gradient: %s", cudaGetErrorString(ej));
    }
    return s;
}

}  // extern "C"
