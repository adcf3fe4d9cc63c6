// autotune.cu -- measured choice of the propagator family for a problem.
//
// Built on the public entry points only: for every family that accepts the
// problem (one CTA per grid, a cluster of CTAs, global-memory tiles, and
// for the CPML absorber its own kernels) and every thread shape of the
// family (fwi_problem.shape: column pairs or single columns for the resident
// kernels, column pairs or 13- or 19-row single-column strips for the cluster
// kernels, 8 or 4 rows a thread or float4 column quads for the tiled kernels) it
// creates plans on two shortened time axes (T and 2T steps), times one
// gradient pass (forward with the record, adjoint) on each after an untimed
// one, in caller-provided scratch, and predicts the pass at the problem's nt
// from the fixed cost and the cost per step the two timings give.  The
// families differ in both: the cluster kernels set up per-CTA tables in
// shared memory once per pass, the tiled kernels launch once per step.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "fwi_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr int kFamilies[4] = {FWI_KERNELS_RESIDENT, FWI_KERNELS_TILED, FWI_KERNELS_CLUSTER,
                               FWI_KERNELS_CPML};
// the shapes tried per family (in kFamilies order), default first
constexpr int kMaxShapes = 3;
constexpr int kShapes[4][kMaxShapes] = {
    {FWI_SHAPE_RESIDENT_PAIRS, FWI_SHAPE_RESIDENT_COLUMNS, -1},
    {FWI_SHAPE_TILED_QUADS, FWI_SHAPE_TILED_ROWS8, FWI_SHAPE_TILED_ROWS4},
    {FWI_SHAPE_CLUSTER_PAIRS, FWI_SHAPE_CLUSTER_RS13, FWI_SHAPE_CLUSTER_RS19},
    {FWI_SHAPE_DEFAULT, -1, -1}};

size_t up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

struct Trial {
    fwi_plan *plan = nullptr;
    size_t ws = 0, snap = 0, data = 0, grad = 0;
    size_t total() const { return up(ws) + up(snap) + up(data) + up(grad); }
};

// Plan of family `fam` for the problem on trial_steps steps; false if the
// family cannot run it (FWI_ERR_UNSUPPORTED), the other errors returned.
fwi_status make_trial(const fwi_problem &p, const fwi_w2_params &w2, int steps, int fam,
                      int shape, Trial *t, bool *ok)
{
    fwi_problem q = p;
    q.nt = steps;
    q.kernels = fam;
    q.shape = shape;
    *ok = false;
    fwi_status s = fwi_plan_create(&q, &w2, &t->plan);
    if (s == FWI_ERR_UNSUPPORTED) return FWI_OK;
    if (s != FWI_OK) return s;
    s = fwi_plan_sizes(t->plan, &t->ws, nullptr, &t->snap);
    if (s != FWI_OK) return s;
    t->data = (size_t)p.batch * p.ns * p.nr * steps * sizeof(float);
    t->grad = (size_t)p.batch * p.nz * p.nx * sizeof(float);
    *ok = true;
    return FWI_OK;
}

fwi_status check_args(const fwi_problem *prob, const fwi_w2_params *w2, int trial_steps)
{
    if (!prob || !w2) return fwi::record_error(FWI_ERR_INVALID_ARG, "problem or w2 params is NULL");
    if (trial_steps < 2 || trial_steps > prob->nt)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "trial_steps must be in [2, nt = %d]",
                                 prob->nt);
    // the problem itself must be valid (any family)
    fwi_problem q = *prob;
    q.kernels = FWI_KERNELS_AUTO;
    q.shape = FWI_SHAPE_DEFAULT;
    fwi_plan *pl = nullptr;
    const fwi_status s = fwi_plan_create(&q, w2, &pl);
    fwi_plan_destroy(pl);
    return s;
}

// The longer of the two trial lengths.
int long_trial(const fwi_problem &p, int trial_steps)
{
    return 2 * trial_steps < p.nt ? 2 * trial_steps : p.nt;
}

}  // namespace

extern "C" {

fwi_status fwi_autotune_scratch_bytes(const fwi_problem *prob, const fwi_w2_params *w2,
                                      int trial_steps, size_t *bytes)
{
    if (!bytes) return fwi::record_error(FWI_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = 0;
    fwi_status s = check_args(prob, w2, trial_steps);
    if (s != FWI_OK) return s;
    for (int k = 0; k < 4; ++k)
        for (int sh : kShapes[k]) {
            if (sh < 0) continue;
            Trial t;
            bool ok = false;
            s = make_trial(*prob, *w2, long_trial(*prob, trial_steps), kFamilies[k], sh, &t, &ok);
            if (ok && t.total() > *bytes) *bytes = t.total();
            fwi_plan_destroy(t.plan);
            if (s != FWI_OK) return s;
        }
    return FWI_OK;
}

fwi_status fwi_autotune_kernels(const fwi_problem *prob, const fwi_w2_params *w2, const float *v,
                                int trial_steps, void *scratch, size_t scratch_bytes,
                                int *family, int *shape, float *ms, int *shapes, void *stream)
{
    if (!v || !scratch || !family || !shape)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "v, scratch, family or shape is NULL");
    fwi_status s = check_args(prob, w2, trial_steps);
    if (s != FWI_OK) return s;
    if ((uintptr_t)scratch % kAlign != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float best = -1.f;
    *family = FWI_KERNELS_AUTO;
    *shape = FWI_SHAPE_DEFAULT;
    float times[4] = {-1.f, -1.f, -1.f, -1.f};
    int best_shape[4] = {-1, -1, -1, -1};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fwi::record_error(FWI_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(ce));
    }
    const int n1 = trial_steps, n2 = long_trial(*prob, trial_steps);
    for (int cand = 0; cand < 4 * kMaxShapes && s == FWI_OK; ++cand) {
        const int k = cand / kMaxShapes, sh = kShapes[k][cand % kMaxShapes];
        if (sh < 0) continue;
        float tl[2] = {-1.f, -1.f};   // best time of one pass at n1 and n2 steps
        bool ran = false;
        for (int L = 0; L < (n2 > n1 ? 2 : 1) && s == FWI_OK; ++L) {
            Trial t;
            bool ok = false;
            s = make_trial(*prob, *w2, L ? n2 : n1, kFamilies[k], sh, &t, &ok);
            if (s == FWI_OK && ok && t.total() > scratch_bytes)
                s = fwi::record_error(FWI_ERR_OOM,
                                      "scratch of %zu bytes < %zu (fwi_autotune_scratch_bytes)",
                                      scratch_bytes, t.total());
            if (s == FWI_OK && ok) {
                unsigned char *base = static_cast<unsigned char *>(scratch);
                void *ws = base;
                float *snap = reinterpret_cast<float *>(base + up(t.ws));
                float *data = reinterpret_cast<float *>(base + up(t.ws) + up(t.snap));
                float *grad =
                    reinterpret_cast<float *>(base + up(t.ws) + up(t.snap) + up(t.data));
                for (int rep = 0; rep < 3 && s == FWI_OK; ++rep) {
                    // rep 0 warms up (first launches, shared-memory carve-out)
                    if (rep > 0 && (ce = cudaEventRecord(e0, st)) != cudaSuccess) break;
                    s = fwi_forward(t.plan, v, data, snap, ws, stream);
                    if (s == FWI_OK) s = fwi_adjoint_grad(t.plan, v, data, snap, grad, ws, stream);
                    if (s != FWI_OK) break;
                    if (rep > 0) {
                        if ((ce = cudaEventRecord(e1, st)) != cudaSuccess) break;
                        if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) break;
                        float m = 0.f;
                        if ((ce = cudaEventElapsedTime(&m, e0, e1)) != cudaSuccess) break;
                        if (tl[L] < 0.f || m < tl[L]) tl[L] = m;
                    }
                }
                if (s == FWI_OK && ce != cudaSuccess)
                    s = fwi::record_error(FWI_ERR_CUDA, "autotune timing: %s",
                                          cudaGetErrorString(ce));
                if (s == FWI_OK) s = fwi_check(t.plan, ws, stream);
                ran = s == FWI_OK;
            }
            fwi_plan_destroy(t.plan);
        }
        if (s == FWI_OK && ran) {
            // predicted pass at nt steps: fixed + nt x per-step cost
            float pred = tl[0];
            if (n2 > n1) {
                float per = (tl[1] - tl[0]) / (float)(n2 - n1);
                if (per < 0.f) per = 0.f;
                pred = tl[0] + per * (float)(prob->nt - n1);
            }
            if (times[k] < 0.f || pred < times[k]) {
                times[k] = pred;
                best_shape[k] = sh;
            }
            if (best < 0.f || pred < best) {
                best = pred;
                *family = kFamilies[k];
                *shape = sh;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms) std::memcpy(ms, times, sizeof(times));
    if (shapes) std::memcpy(shapes, best_shape, sizeof(best_shape));
    if (s == FWI_OK) fwi::record_error(FWI_OK, "%s", "");   // families that declined left a message
    return s;
}

}  // extern "C"
