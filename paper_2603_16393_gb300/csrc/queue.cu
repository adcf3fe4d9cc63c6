// queue.cu -- forward and adjoint passes of several plans of uneven grid sizes
// in one persistent launch each: the (model, shot) units of every plan go on
// one numbered list (the plans in the caller's order, largest first for the
// best balance), and every CTA of the column-pair propagators draws the next
// unit from a counter in device memory until the list is done, so one launch
// runs units of different grids side by side and no SM idles in the tail of
// one plan while another's units wait.
#include <cuda_runtime.h>

#include <cstdint>

#include "fwi_internal.cuh"

namespace {

// lists: nl per-plan pointer lists, none may hold NULL; bit l of align16 set:
// list l's pointers must be 16-byte aligned (record planes, workspace)
fwi_status check_plans(const fwi_plan *const *plans, int n, const void *const *lists[], int nl,
                       unsigned align16, int *counter, const char *what)
{
    if (!plans || n < 1 || n > fwi::kQueuePlans)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "%s: need 1 <= n <= %d plans", what,
                                 fwi::kQueuePlans);
    if (!counter) return fwi::record_error(FWI_ERR_INVALID_ARG, "%s: counter is NULL", what);
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fwi::record_error(FWI_ERR_INVALID_ARG, "%s: plan %d is NULL", what, i);
        for (int l = 0; l < nl; ++l) {
            if (!lists[l] || !lists[l][i])
                return fwi::record_error(FWI_ERR_INVALID_ARG, "%s: a pointer of plan %d is NULL",
                                         what, i);
            if (((align16 >> l) & 1u) && (reinterpret_cast<uintptr_t>(lists[l][i]) & 15u) != 0)
                return fwi::record_error(FWI_ERR_INVALID_ARG,
                                         "%s: a pointer of plan %d is not 16-byte aligned", what,
                                         i);
        }
        const fwi::Plan &pl = *reinterpret_cast<const fwi::Plan *>(plans[i]);
        if (!fwi::queue_ok(pl))
            return fwi::record_error(FWI_ERR_UNSUPPORTED,
                                     "%s: plan %d is not a store-all plan of the resident "
                                     "column-pair kernels (padded grid NZ <= 110, even NX <= 156)",
                                     what, i);
        const fwi::Plan &p0 = *reinterpret_cast<const fwi::Plan *>(plans[0]);
        if (!fwi::queue_same_physics(pl, p0))
            return fwi::record_error(FWI_ERR_UNSUPPORTED,
                                     "%s: plan %d differs from plan 0 in dx, dz, dt, nb, top_bc, "
                                     "v_ref, refl_R or the source wavelet",
                                     what, i);
    }
    return FWI_OK;
}

void full_window(fwi::PropArgs &a)
{
    a.j_begin = 0;
    a.j_end = a.nt;
    a.rec_base = 0;
    a.rec_planes = a.nt;
}

}  // namespace

extern "C" {

fwi_status fwi_queue_forward(const fwi_plan *const *plans, int n, const float *const *v,
                             float *const *d_syn, float *const *snapshots,
                             void *const *workspace, int *counter, void *stream)
{
    const void *const *lists[] = {(const void *const *)v, (const void *const *)d_syn,
                                  (const void *const *)snapshots, (const void *const *)workspace};
    fwi_status s = check_plans(plans, n, lists, 4, 0xcu, counter, "fwi_queue_forward");
    if (s != FWI_OK) return s;
    const fwi::Plan *pls[fwi::kQueuePlans];
    fwi::PropArgs a[fwi::kQueuePlans];
    for (int i = 0; i < n; ++i) {
        pls[i] = reinterpret_cast<const fwi::Plan *>(plans[i]);
        a[i] = fwi::make_args(*pls[i]);
        a[i].v = v[i];
        a[i].d_syn = d_syn[i];
        a[i].snap = snapshots[i];
        a[i].status = static_cast<int *>(workspace[i]);
        full_window(a[i]);
    }
    const cudaError_t e =
        fwi::launch_fast_queue(pls, n, false, a, counter, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_queue_forward launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_queue_adjoint(const fwi_plan *const *plans, int n, const float *const *v,
                             const float *const *adj_src, const float *const *snapshots,
                             float *const *grad, void *const *workspace, int *counter,
                             void *stream)
{
    const void *const *lists[] = {(const void *const *)v, (const void *const *)adj_src,
                                  (const void *const *)snapshots, (const void *const *)grad,
                                  (const void *const *)workspace};
    fwi_status s = check_plans(plans, n, lists, 5, 0x14u, counter, "fwi_queue_adjoint");
    if (s != FWI_OK) return s;
    const fwi::Plan *pls[fwi::kQueuePlans];
    fwi::PropArgs a[fwi::kQueuePlans];
    for (int i = 0; i < n; ++i) {
        pls[i] = reinterpret_cast<const fwi::Plan *>(plans[i]);
        a[i] = fwi::make_args(*pls[i]);
        a[i].v = v[i];
        a[i].adj = adj_src[i];
        a[i].snap = const_cast<float *>(snapshots[i]);
        unsigned char *ws = static_cast<unsigned char *>(workspace[i]);
        a[i].gshot = reinterpret_cast<float *>(ws + pls[i]->ws_gshot);
        a[i].status = reinterpret_cast<int *>(ws);
        full_window(a[i]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = fwi::launch_fast_queue(pls, n, true, a, counter, st);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const fwi::Plan &pl = *pls[i];
        const int cells = pl.p.nz * pl.p.nx;
        const dim3 grid((cells + 255) / 256, pl.p.batch);
        fwi::k_shot_sum<<<grid, 256, 0, st>>>(pl.p.batch, pl.p.ns, cells, a[i].gshot, grad[i]);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_queue_adjoint launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

}  // extern "C"
