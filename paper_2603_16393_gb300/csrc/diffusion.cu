// diffusion.cu -- the elementwise steps of one reverse step i -> i-1 of
// Algorithm 1 (DPS) and Algorithm 2 (OT-guided preconditioned DPS) around the
// physics gradient, each one pass over [B][ncell]:
//   k_ddpm_proposal: score (given, or of a Gaussian prior), the clean
//     estimate of Eq. v0hat, the prior-driven proposal v' of Algorithms 1-2,
//     and the clamped physical model the propagators run on;
//   k_ddpm_guidance: dPhi/dv0hat in the normalised space and, by
//     Eq. chain_rule, dPhi/dv_i through the clean estimate.
// The per-step coefficients are formed on the host in FP64 and rounded once;
// 1 - abar_i is never formed in float32 (it is 1e-4 at i = 1).
//
// Gaussian prior (x_0 ~ N(mu, tau2)): Eq. v0hat and Eq. chain_rule as written
// cancel at high noise (x + (1 - abar) s -> 0 while 1/sqrt(abar) -> 160 at
// abar = 4e-5, and 1 - (1 - abar)/D -> abar tau2 / D), so the prior path
// evaluates the same quantities in their cancellation-free closed forms,
// with D = abar tau2 + 1 - abar:
//   v0hat = (sqrt(abar) tau2 x + (1 - abar) mu) / D   (Tweedie's mean)
//   h     = sqrt(abar) tau2 g / D
// A caller's score goes through Eq. v0hat and Eq. chain_rule as written.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "fwi_internal.cuh"

namespace {

constexpr int kThreads = 256;

struct StepF {
    float abar, one_m_abar, sqrt_abar, inv_sqrt_abar;
    float c_v, c_0, sigma;
    float shift, unit, v_lo, v_hi;
};

StepF step_f(const fwi_ddpm_step &s, const fwi_diffusion_space &sp)
{
    StepF k;
    k.abar = (float)s.abar;
    k.one_m_abar = (float)(1.0 - s.abar);
    k.sqrt_abar = (float)std::sqrt(s.abar);
    k.inv_sqrt_abar = (float)(1.0 / std::sqrt(s.abar));
    k.c_v = (float)s.c_v;
    k.c_0 = (float)s.c_0;
    k.sigma = (float)s.sigma;
    k.shift = (float)sp.shift;
    k.unit = (float)sp.unit;
    k.v_lo = (float)sp.v_lo;
    k.v_hi = (float)sp.v_hi;
    return k;
}

// Eq. v0hat with the prior's score s = -(x - sqrt(abar) mu) / D, the score of
// the step-i marginal N(sqrt(abar) mu, D) of N(mu, tau2)
__device__ __forceinline__ float prior_clean_estimate(float x, float mu, float tau2,
                                                      const StepF &k)
{
    const float D = fmaf(k.abar, tau2, k.one_m_abar);
    return __fdiv_rn(fmaf(k.sqrt_abar * tau2, x, k.one_m_abar * mu), D);
}

// IDX: 32-bit element indices (and cell modulo) when B ncell < 2^32
// DEV: the coefficients are record *step of the device table and the draws
// are z + *step z_stride (a reverse step whose launches replay from a CUDA
// graph); an index outside 1..n_steps writes nothing
template <typename IDX, bool DEV>
__global__ void __launch_bounds__(kThreads)
    k_ddpm_proposal(IDX n, IDX ncell, StepF kv, const float *__restrict__ table,
                    const int *__restrict__ step, int n_steps, size_t z_stride,
                    const float *__restrict__ v_i,
                    const float *__restrict__ score, const float *__restrict__ mu,
                    const float *__restrict__ tau2, const float *__restrict__ z,
                    float *__restrict__ v0hat, float *__restrict__ v_prime,
                    float *__restrict__ v_phys)
{
    StepF k = kv;
    if (DEV) {
        const int i = *step;
        if (i < 1 || i > n_steps) return;
        k = *reinterpret_cast<const StepF *>(table + (size_t)i * FWI_DDPM_RECORD_FLOATS);
        z += (size_t)i * z_stride;
    }
    for (IDX e = (IDX)blockIdx.x * kThreads + threadIdx.x; e < n; e += (IDX)gridDim.x * kThreads) {
        const float x = v_i[e];
        float x0;
        if (score) {
            x0 = fmaf(k.one_m_abar, score[e], x) * k.inv_sqrt_abar;     // Eq. v0hat
        } else {
            const IDX c = e % ncell;
            x0 = prior_clean_estimate(x, mu[c], tau2[c], k);
        }
        v0hat[e] = x0;
        v_prime[e] = fmaf(k.c_v, x, fmaf(k.c_0, x0, k.sigma * z[e]));
        v_phys[e] = fminf(fmaxf(fmaf(k.unit, x0, k.shift), k.v_lo), k.v_hi);
    }
}

template <typename IDX, bool DEV>
__global__ void __launch_bounds__(kThreads)
    k_ddpm_guidance(IDX n, IDX ncell, StepF kv, const float *__restrict__ table,
                    const int *__restrict__ step, int n_steps, const float *__restrict__ v0hat,
                    const float *__restrict__ g_phys, const float *__restrict__ vjp,
                    const float *__restrict__ tau2, float *__restrict__ g,
                    float *__restrict__ h)
{
    StepF k = kv;
    if (DEV) {
        const int i = *step;
        if (i < 1 || i > n_steps) return;
        k = *reinterpret_cast<const StepF *>(table + (size_t)i * FWI_DDPM_RECORD_FLOATS);
    }
    for (IDX e = (IDX)blockIdx.x * kThreads + threadIdx.x; e < n; e += (IDX)gridDim.x * kThreads) {
        // the clamp passes the gradient only where it is the identity
        const float vp = fmaf(k.unit, v0hat[e], k.shift);
        const float gg = (vp >= k.v_lo && vp <= k.v_hi) ? k.unit * g_phys[e] : 0.f;
        float hh;
        if (vjp) {
            hh = fmaf(k.one_m_abar, vjp[e], gg) * k.inv_sqrt_abar;     // Eq. chain_rule
        } else if (tau2) {
            const float t2 = tau2[e % ncell];
            hh = __fdiv_rn(k.sqrt_abar * t2 * gg, fmaf(k.abar, t2, k.one_m_abar));
        } else {
            hh = gg * k.inv_sqrt_abar;                                  // score free of v_i
        }
        g[e] = gg;
        h[e] = hh;
    }
}

unsigned grid_for(size_t n)
{
    // enough CTAs to keep every SM's loads in flight, one grid-stride pass
    // for the sizes the sampler runs (B x 4900 cells)
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n + kThreads - 1) / kThreads;
    const size_t cap = (size_t)sms * 8;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

__global__ void k_step_down(int *step) { *step -= 1; }

// Low-rank Gaussian prior, step i = *step (nothing is written outside 1..N):
// with r = x - sqrt(abar) mu (x alone when mu is NULL), the projections
// p_j = U_j . r scaled by 1/c_j - 1/c_perp,
//   c_j = abar (lam_j + s2) + 1 - abar,  c_perp = abar s2 + 1 - abar.
// One CTA per (model, direction); per-thread strided sums, then a fixed
// tree: the same bits on every call.
__global__ void __launch_bounds__(kThreads)
    k_lr_project(int ncell, int k, const float *__restrict__ U, const float *__restrict__ lam,
                 float s2, const float *__restrict__ x, const float *__restrict__ mu,
                 const float *__restrict__ table, const int *__restrict__ step, int n_steps,
                 float *__restrict__ q)
{
    __shared__ float red[kThreads];
    const int i = *step;
    if (i < 1 || i > n_steps) return;
    const float *rec = table + (size_t)i * FWI_DDPM_RECORD_FLOATS;
    const float abar = rec[0], one_m_abar = rec[1], sqrt_abar = rec[2];
    const int b = blockIdx.x, j = blockIdx.y;
    const float *xb = x + (size_t)b * ncell, *Uj = U + (size_t)j * ncell;
    float acc = 0.f;
    for (int e = threadIdx.x; e < ncell; e += kThreads) {
        const float r = mu ? fmaf(-sqrt_abar, mu[e], xb[e]) : xb[e];
        acc = fmaf(Uj[e], r, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float cj = fmaf(abar, lam[j] + s2, one_m_abar);
        const float cp = fmaf(abar, s2, one_m_abar);
        q[(size_t)b * k + j] = red[0] * (__fdiv_rn(1.f, cj) - __fdiv_rn(1.f, cp));
    }
}

// out = -(r / c_perp + sum_j q_j U_j): the score of the step-i marginal at x
// (mu given), or -C^-1 x, its vector-Jacobian product applied to x (mu NULL)
__global__ void __launch_bounds__(kThreads)
    k_lr_apply(int batch, int ncell, int k, const float *__restrict__ U, float s2,
               const float *__restrict__ x, const float *__restrict__ mu,
               const float *__restrict__ q, const float *__restrict__ table,
               const int *__restrict__ step, int n_steps, float *__restrict__ out)
{
    const int i = *step;
    if (i < 1 || i > n_steps) return;
    const float *rec = table + (size_t)i * FWI_DDPM_RECORD_FLOATS;
    const float abar = rec[0], one_m_abar = rec[1], sqrt_abar = rec[2];
    const float cp = fmaf(abar, s2, one_m_abar);
    const size_t n = (size_t)batch * ncell;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const int c = (int)(e % ncell);
        const size_t b = e / ncell;
        const float r = mu ? fmaf(-sqrt_abar, mu[c], x[e]) : x[e];
        float acc = 0.f;
        const float *qb = q + b * k;
        for (int j = 0; j < k; ++j) acc = fmaf(qb[j], U[(size_t)j * ncell + c], acc);
        out[e] = -(__fdiv_rn(r, cp) + acc);
    }
}

bool finite(double x) { return std::isfinite(x); }

static_assert(sizeof(StepF) == FWI_DDPM_RECORD_FLOATS * sizeof(float) - sizeof(float),
              "a table record is one StepF and one float of padding");

fwi_status check_space(const fwi_diffusion_space *space)
{
    if (!space) return fwi::record_error(FWI_ERR_INVALID_ARG, "space must not be NULL");
    const fwi_diffusion_space &sp = *space;
    if (!finite(sp.shift) || !(sp.unit > 0.0) || !finite(sp.unit) || !finite(sp.v_lo) ||
        !finite(sp.v_hi) || !(sp.v_lo < sp.v_hi))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "need finite shift, unit > 0 and finite v_lo < v_hi");
    return FWI_OK;
}

fwi_status check_common(int batch, int ncell, const fwi_ddpm_step *step,
                        const fwi_diffusion_space *space)
{
    if (batch < 1 || ncell < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "batch and ncell must be >= 1");
    if (!step || !space)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "step and space must not be NULL");
    const fwi_ddpm_step &s = *step;
    if (!(s.abar > 0.0 && s.abar < 1.0) || !finite(s.c_v) || !finite(s.c_0) ||
        !(s.sigma >= 0.0) || !finite(s.sigma))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "need 0 < abar < 1, finite c_v, c_0 and sigma >= 0");
    const fwi_diffusion_space &sp = *space;
    if (!finite(sp.shift) || !(sp.unit > 0.0) || !finite(sp.unit) || !finite(sp.v_lo) ||
        !finite(sp.v_hi) || !(sp.v_lo < sp.v_hi))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "need finite shift, unit > 0 and finite v_lo < v_hi");
    return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_ddpm_coefficients(const double *betas, int n_steps, int i, int sigma_mode,
                                 fwi_ddpm_step *out)
{
    if (!betas || !out) return fwi::record_error(FWI_ERR_INVALID_ARG, "betas and out must not be NULL");
    if (n_steps < 1 || i < 1 || i > n_steps)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "need 1 <= i <= n_steps (i = %d, n = %d)",
                                 i, n_steps);
    if (sigma_mode != FWI_SIGMA_POSTERIOR && sigma_mode != FWI_SIGMA_BETA)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "sigma_mode must be 0 or 1");
    double abar_prev = 1.0, abar = 1.0;   // abar_0 = 1
    for (int j = 1; j <= i; ++j) {
        const double b = betas[j - 1];
        if (!(b > 0.0 && b < 1.0))
            return fwi::record_error(FWI_ERR_INVALID_ARG, "beta_%d = %g is not in (0, 1)", j, b);
        abar_prev = abar;
        abar = abar * (1.0 - b);
    }
    const double beta = betas[i - 1];
    out->abar = abar;
    out->c_v = std::sqrt(1.0 - beta) * (1.0 - abar_prev) / (1.0 - abar);
    out->c_0 = std::sqrt(abar_prev) * beta / (1.0 - abar);
    out->sigma = sigma_mode == FWI_SIGMA_POSTERIOR
                     ? std::sqrt((1.0 - abar_prev) * beta / (1.0 - abar))
                     : std::sqrt(beta);
    return FWI_OK;
}

fwi_status fwi_ddpm_proposal(int batch, int ncell, const fwi_ddpm_step *step,
                             const fwi_diffusion_space *space, const float *v_i,
                             const float *score, const float *mu, const float *tau2,
                             const float *z, float *v0hat, float *v_prime, float *v_phys,
                             void *stream)
{
    fwi_status s = check_common(batch, ncell, step, space);
    if (s != FWI_OK) return s;
    if (!v_i || !z || !v0hat || !v_prime || !v_phys)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "v_i, z and the outputs must not be NULL");
    if (!score && (!mu || !tau2))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "without a score, mu and tau2 are needed");
    const size_t n = (size_t)batch * (size_t)ncell;
    const StepF k = step_f(*step, *space);
    cudaStream_t st = (cudaStream_t)stream;
    if (n + (size_t)grid_for(n) * kThreads < ((size_t)1 << 32))
        k_ddpm_proposal<unsigned, false><<<grid_for(n), kThreads, 0, st>>>(
            (unsigned)n, (unsigned)ncell, k, nullptr, nullptr, 0, 0, v_i, score, mu, tau2, z,
            v0hat, v_prime, v_phys);
    else
        k_ddpm_proposal<size_t, false><<<grid_for(n), kThreads, 0, st>>>(
            n, (size_t)ncell, k, nullptr, nullptr, 0, 0, v_i, score, mu, tau2, z, v0hat, v_prime,
            v_phys);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_ddpm_proposal launch: %s", cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_ddpm_guidance(int batch, int ncell, const fwi_ddpm_step *step,
                             const fwi_diffusion_space *space, const float *v0hat,
                             const float *g_phys, const float *vjp, const float *tau2, float *g,
                             float *h, void *stream)
{
    fwi_status s = check_common(batch, ncell, step, space);
    if (s != FWI_OK) return s;
    if (!v0hat || !g_phys || !g || !h)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "v0hat, g_phys, g and h must not be NULL");
    const size_t n = (size_t)batch * (size_t)ncell;
    const StepF k = step_f(*step, *space);
    cudaStream_t st = (cudaStream_t)stream;
    if (n + (size_t)grid_for(n) * kThreads < ((size_t)1 << 32))
        k_ddpm_guidance<unsigned, false><<<grid_for(n), kThreads, 0, st>>>(
            (unsigned)n, (unsigned)ncell, k, nullptr, nullptr, 0, v0hat, g_phys, vjp, tau2, g, h);
    else
        k_ddpm_guidance<size_t, false><<<grid_for(n), kThreads, 0, st>>>(
            n, (size_t)ncell, k, nullptr, nullptr, 0, v0hat, g_phys, vjp, tau2, g, h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_ddpm_guidance launch: %s", cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_ddpm_table(const double *betas, int n_steps, int sigma_mode,
                          const fwi_diffusion_space *space, float *table)
{
    if (!table) return fwi::record_error(FWI_ERR_INVALID_ARG, "table must not be NULL");
    fwi_status s = check_space(space);
    if (s != FWI_OK) return s;
    float *rec = table;
    for (int f = 0; f < FWI_DDPM_RECORD_FLOATS; ++f) rec[f] = 0.f;   // record 0 is unused
    for (int i = 1; i <= n_steps; ++i) {
        fwi_ddpm_step st;
        s = fwi_ddpm_coefficients(betas, n_steps, i, sigma_mode, &st);
        if (s != FWI_OK) return s;
        const StepF k = step_f(st, *space);
        float *r = table + (size_t)i * FWI_DDPM_RECORD_FLOATS;
        std::memcpy(r, &k, sizeof(StepF));
        r[FWI_DDPM_RECORD_FLOATS - 1] = 0.f;
    }
    return FWI_OK;
}

fwi_status fwi_ddpm_proposal_at(int batch, int ncell, const float *table, const int *step,
                                int n_steps, const float *v_i, const float *score,
                                const float *mu, const float *tau2, const float *z,
                                long long z_stride, float *v0hat, float *v_prime, float *v_phys,
                                void *stream)
{
    if (batch < 1 || ncell < 1 || n_steps < 1 || z_stride < 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "batch, ncell, n_steps >= 1 and z_stride >= 0 needed");
    if (!table || !step || !v_i || !z || !v0hat || !v_prime || !v_phys)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "table, step, v_i, z and the outputs must not be NULL");
    if (!score && (!mu || !tau2))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "without a score, mu and tau2 are needed");
    const size_t n = (size_t)batch * (size_t)ncell;
    const float *tab = table;
    static_assert(alignof(StepF) == alignof(float), "records are float arrays");
    cudaStream_t st = (cudaStream_t)stream;
    if (n + (size_t)grid_for(n) * kThreads < ((size_t)1 << 32))
        k_ddpm_proposal<unsigned, true><<<grid_for(n), kThreads, 0, st>>>(
            (unsigned)n, (unsigned)ncell, StepF{}, tab, step, n_steps, (size_t)z_stride, v_i,
            score, mu, tau2, z, v0hat, v_prime, v_phys);
    else
        k_ddpm_proposal<size_t, true><<<grid_for(n), kThreads, 0, st>>>(
            n, (size_t)ncell, StepF{}, tab, step, n_steps, (size_t)z_stride, v_i, score, mu, tau2,
            z, v0hat, v_prime, v_phys);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_ddpm_proposal_at launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_ddpm_guidance_at(int batch, int ncell, const float *table, const int *step,
                                int n_steps, const float *v0hat, const float *g_phys,
                                const float *vjp, const float *tau2, float *g, float *h,
                                void *stream)
{
    if (batch < 1 || ncell < 1 || n_steps < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "batch, ncell, n_steps must be >= 1");
    if (!table || !step || !v0hat || !g_phys || !g || !h)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "table, step, v0hat, g_phys, g and h must not be NULL");
    const size_t n = (size_t)batch * (size_t)ncell;
    const float *tab = table;
    cudaStream_t st = (cudaStream_t)stream;
    if (n + (size_t)grid_for(n) * kThreads < ((size_t)1 << 32))
        k_ddpm_guidance<unsigned, true><<<grid_for(n), kThreads, 0, st>>>(
            (unsigned)n, (unsigned)ncell, StepF{}, tab, step, n_steps, v0hat, g_phys, vjp, tau2,
            g, h);
    else
        k_ddpm_guidance<size_t, true><<<grid_for(n), kThreads, 0, st>>>(
            n, (size_t)ncell, StepF{}, tab, step, n_steps, v0hat, g_phys, vjp, tau2, g, h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_ddpm_guidance_at launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_ddpm_step_down(int *step, void *stream)
{
    if (!step) return fwi::record_error(FWI_ERR_INVALID_ARG, "step must not be NULL");
    k_step_down<<<1, 1, 0, (cudaStream_t)stream>>>(step);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_ddpm_step_down launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

fwi_status fwi_lowrank_score_at(int batch, int ncell, int k, const float *U, const float *lam,
                                double s2, const float *x, const float *mu, const float *table,
                                const int *step, int n_steps, float *work, float *out,
                                void *stream)
{
    if (batch < 1 || ncell < 1 || k < 0 || k > 65535 || n_steps < 1 || !(s2 > 0.0) ||
        !std::isfinite(s2))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "batch, ncell, n_steps >= 1, 0 <= k <= 65535 and s2 > 0 needed");
    if (!x || !table || !step || !out || (k > 0 && (!U || !lam || !work)))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "x, table, step, out (and U, lam, work when k > 0) must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (k > 0)
        k_lr_project<<<dim3((unsigned)batch, (unsigned)k), kThreads, 0, st>>>(
            ncell, k, U, lam, (float)s2, x, mu, table, step, n_steps, work);
    const size_t n = (size_t)batch * (size_t)ncell;
    k_lr_apply<<<grid_for(n), kThreads, 0, st>>>(batch, ncell, k, U, (float)s2, x, mu, work,
                                                 table, step, n_steps, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_lowrank_score_at launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

}  // extern "C"
