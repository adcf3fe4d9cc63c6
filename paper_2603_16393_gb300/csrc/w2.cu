// w2.cu -- weighted, normalised Wasserstein-2 misfit (Sec. 5.1, 6.2) and its
// exact derivative, one CTA per trace.
//
// Per trace (Sec. 6.2 numerics):
//   y = omega d + c',  Z = dt (sum y - (y_0 + y_{nt-1})/2),  p = y / (Z + eps')
//   F_0 = 0, F_k = F_{k-1} + dt (p_{k-1} + p_k)/2          (block prefix scan)
//   k*_j = min{k : F_k >= xi_j} = lower_bound of the running max of F
//   Q_j = t_{k*-1} + dt (xi_j - F_{k*-1}) / (F_{k*} - F_{k*-1}), clamped at the ends
//   W2 = (dxi sum_j w_j (Q_j - Qobs_j)^2)^(1/2),  J = sum W2 / S_obs
// Reverse pass without scatter: with a_j, b_j the contributions of node j to
// dJ/dF_{k*-1} and dJ/dF_{k*}, and k*_j non-decreasing in j,
//   H_k = sum_{k' >= k} dJ/dF_{k'} = SA[J(k+1)] + SB[J(k)],
// where SA, SB are suffix sums over j and J(k) = min{j : k*_j >= k}; then
//   dJ/dp_m = dt/2 (H_m [m >= 1] + H_{m+1}),
//   dJ/dy_m = dJ/dp_m / (Z+eps') - (sum_n dJ/dp_n y_n) dt w'_m / (Z+eps')^2,
//   dJ/dd_m = omega_m dJ/dy_m.
// Every reduction has a fixed order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int NT_W2 = 256;          // threads per trace CTA
constexpr int NW_W2 = NT_W2 / 32;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- block helpers
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// op: 0 sum, 1 max, 2 min.  Result broadcast to every thread.
template <int OP, int NTH>
__device__ float block_reduce(float v, float *red)
{
    constexpr int NW = NTH / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = OP == 0 ? warp_sum(v) : OP == 1 ? warp_max(v) : warp_min(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float u = lane < NW ? red[lane] : (OP == 0 ? 0.f : OP == 1 ? -INFINITY : INFINITY);
        u = OP == 0 ? warp_sum(u) : OP == 1 ? warp_max(u) : warp_min(u);
        if (lane == 0) red[NW] = u;
    }
    __syncthreads();
    return red[NW];
}

// In-place inclusive scan (OP 0: sum, 1: max) of arr[0..n) in shared memory,
// blocked arrangement (thread t owns a contiguous run).  If REV, the scan runs
// from the end (suffix scan).
template <int OP, bool REV>
__device__ void block_scan(float *arr, int n, float *red)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int per = (n + NT_W2 - 1) / NT_W2;
    const int lo = tid * per, hi = min(lo + per, n);
    const float ident = OP == 0 ? 0.f : -INFINITY;
    float run = ident;
    for (int i = lo; i < hi; ++i) {
        const int k = REV ? n - 1 - i : i;
        run = OP == 0 ? run + arr[k] : fmaxf(run, arr[k]);
        arr[k] = run;
    }
    float incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl = OP == 0 ? incl + y : fmaxf(incl, y);
    }
    __syncthreads();
    if (lane == 31) red[w] = incl;
    __syncthreads();
    if (w == 0) {
        float u = lane < NW_W2 ? red[lane] : ident;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(FULL, u, o);
            if (lane >= o) u = OP == 0 ? u + y : fmaxf(u, y);
        }
        if (lane < NW_W2) red[lane] = u;
    }
    __syncthreads();
    // exclusive prefix of this thread = warp-exclusive part + previous warps
    const float prev_in_warp = __shfl_up_sync(FULL, incl, 1);
    float off = (lane > 0) ? prev_in_warp : ident;
    if (w > 0) off = (lane > 0) ? (OP == 0 ? off + red[w - 1] : fmaxf(off, red[w - 1])) : red[w - 1];
    if (tid > 0) {
        for (int i = lo; i < hi; ++i) {
            const int k = REV ? n - 1 - i : i;
            arr[k] = OP == 0 ? arr[k] + off : fmaxf(arr[k], off);
        }
    }
    __syncthreads();
}

// first k in [0, n) with a[k] >= x for non-decreasing a; n if none
__device__ __forceinline__ int lower_bound_f(const float *a, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound_i(const int *a, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct CtxPtrs {
    float *M, *S, *cshift, *s_tr, *omega, *Q;
};

inline CtxPtrs ctx_ptrs(const Plan &pl, unsigned char *ctx)
{
    CtxPtrs c;
    c.M = (float *)(ctx + pl.ctx_M);
    c.S = (float *)(ctx + pl.ctx_S);
    c.cshift = (float *)(ctx + pl.ctx_cshift);
    c.s_tr = (float *)(ctx + pl.ctx_str);
    c.omega = (float *)(ctx + pl.ctx_omega);
    c.Q = (float *)(ctx + pl.ctx_Q);
    return c;
}

struct W2Args {
    int nt, nxi, ntr;           // ntr = ns * nr traces per instance
    float dt, k, cfac, eps;
    CtxPtrs c;
};

// y (in smem) holds omega*d + c'; builds p -> F (in place into F), the running
// max Fm, and returns Z.
__device__ float density_cdf(const float *y, float *F, float *Fm, int nt, float dt, float eps,
                             float *red)
{
    float part = 0.f;
    for (int i = threadIdx.x; i < nt; i += NT_W2) part += y[i];
    const float sum = block_reduce<0, NT_W2>(part, red);
    const float Z = dt * (sum - 0.5f * (y[0] + y[nt - 1]));
    const float inv = 1.f / (Z + eps);
    // increments of the trapezoid CDF
    for (int i = threadIdx.x; i < nt; i += NT_W2)
        F[i] = (i == 0) ? 0.f : 0.5f * dt * (y[i - 1] + y[i]) * inv;
    __syncthreads();
    block_scan<0, false>(F, nt, red);
    for (int i = threadIdx.x; i < nt; i += NT_W2) Fm[i] = F[i];
    __syncthreads();
    block_scan<1, false>(Fm, nt, red);
    return Z;
}

// quantile of node j; writes k*
__device__ __forceinline__ float quantile(const float *F, const float *Fm, int nt, float dt,
                                          float xi, int *kst)
{
    const int k = lower_bound_f(Fm, nt, xi);
    *kst = k;
    if (k == 0) return 0.f;
    if (k == nt) return (float)(nt - 1) * dt;
    return (float)(k - 1) * dt + dt * (xi - F[k - 1]) / (F[k] - F[k - 1]);
}

// ------------------------------------------------------------------ kernels
// M[b] = max |d_obs| over the instance
__global__ void __launch_bounds__(1024) k_obs_max(const float *__restrict__ d, size_t per_inst,
                                                  float *__restrict__ M)
{
    __shared__ float red[40];
    const float *db = d + (size_t)blockIdx.x * per_inst;
    float m = 0.f;
    for (size_t i = threadIdx.x; i < per_inst; i += blockDim.x) m = fmaxf(m, fabsf(db[i]));
    m = block_reduce<1, 1024>(m, red);
    if (threadIdx.x == 0) M[blockIdx.x] = m;
}

__global__ void __launch_bounds__(NT_W2) k_obs_trace(const float *__restrict__ d_obs, W2Args a)
{
    extern __shared__ float smw[];
    __shared__ float red[NW_W2 + 2];
    const int tr_g = blockIdx.x;                 // b * ntr + tr
    const int b = tr_g / a.ntr;
    float *y = smw, *F = y + a.nt, *Fm = F + a.nt;
    const float *d = d_obs + (size_t)tr_g * a.nt;
    float *om = a.c.omega + (size_t)tr_g * a.nt;
    const float M = a.c.M[b];
    float mn = INFINITY;
    for (int i = threadIdx.x; i < a.nt; i += NT_W2) {
        const float di = d[i];
        const float w = 1.f / (1.f + a.k * (M > 0.f ? fabsf(di) / M : 0.f));
        om[i] = w;
        const float yi = w * di;
        y[i] = yi;
        mn = fminf(mn, yi);
    }
    mn = block_reduce<2, NT_W2>(mn, red);
    const float cs = a.cfac * fabsf(mn);
    if (threadIdx.x == 0) a.c.cshift[tr_g] = cs;
    for (int i = threadIdx.x; i < a.nt; i += NT_W2) y[i] += cs;
    __syncthreads();
    density_cdf(y, F, Fm, a.nt, a.dt, a.eps, red);
    float *Q = a.c.Q + (size_t)tr_g * a.nxi;
    const float inv = 1.f / (float)(a.nxi - 1);
    float part = 0.f;
    for (int j = threadIdx.x; j < a.nxi; j += NT_W2) {
        const float xi = (float)j / (float)(a.nxi - 1);
        int ks;
        const float q = quantile(F, Fm, a.nt, a.dt, xi, &ks);
        Q[j] = q;
        const float wj = (j == 0 || j == a.nxi - 1) ? 0.5f : 1.f;
        part += wj * q * q;
    }
    const float s2 = block_reduce<0, NT_W2>(part, red);
    if (threadIdx.x == 0) a.c.s_tr[tr_g] = sqrtf(inv * s2);
}

// S[b] = sum of the per-trace scales (fixed order)
__global__ void __launch_bounds__(NT_W2) k_sum_traces(const float *__restrict__ v, int ntr,
                                                      const float *__restrict__ div,
                                                      float *__restrict__ out)
{
    __shared__ float red[NW_W2 + 2];
    const float *vb = v + (size_t)blockIdx.x * ntr;
    float part = 0.f;
    for (int i = threadIdx.x; i < ntr; i += NT_W2) part += vb[i];
    const float s = block_reduce<0, NT_W2>(part, red);
    if (threadIdx.x == 0) out[blockIdx.x] = div ? s / div[blockIdx.x] : s;
}

__global__ void __launch_bounds__(NT_W2) k_misfit_trace(const float *__restrict__ d_syn, W2Args a,
                                                        float *__restrict__ w2_dst,
                                                        float *__restrict__ adj)
{
    extern __shared__ float smw[];
    __shared__ float red[NW_W2 + 2];
    const int tr_g = blockIdx.x;
    const int b = tr_g / a.ntr;
    const int nt = a.nt, nxi = a.nxi;
    float *y = smw, *F = y + nt, *Fm = F + nt;
    float *dq = Fm + nt, *A = dq + nxi, *Bq = A + nxi;
    int *ks = (int *)(Bq + nxi);
    const float *d = d_syn + (size_t)tr_g * nt;
    const float *om = a.c.omega + (size_t)tr_g * nt;
    const float cs = a.c.cshift[tr_g];
    for (int i = threadIdx.x; i < nt; i += NT_W2) y[i] = om[i] * d[i] + cs;
    __syncthreads();
    const float Z = density_cdf(y, F, Fm, nt, a.dt, a.eps, red);
    const float *Qo = a.c.Q + (size_t)tr_g * nxi;
    const float dxi = 1.f / (float)(nxi - 1);
    float part = 0.f;
    for (int j = threadIdx.x; j < nxi; j += NT_W2) {
        const float xi = (float)j / (float)(nxi - 1);
        int k;
        const float q = quantile(F, Fm, nt, a.dt, xi, &k);
        const float diff = q - Qo[j];
        dq[j] = diff;
        ks[j] = k;
        const float wj = (j == 0 || j == nxi - 1) ? 0.5f : 1.f;
        part += wj * diff * diff;
    }
    const float W2 = sqrtf(dxi * block_reduce<0, NT_W2>(part, red));
    if (threadIdx.x == 0) w2_dst[tr_g] = W2;
    if (!adj) return;
    float *ad = adj + (size_t)tr_g * nt;
    if (W2 == 0.f) {   // non-differentiable point: zero adjoint source
        for (int i = threadIdx.x; i < nt; i += NT_W2) ad[i] = 0.f;
        return;
    }
    const float scale = dxi / (W2 * a.c.S[b]);
    for (int j = threadIdx.x; j < nxi; j += NT_W2) {
        const int k = ks[j];
        float aj = 0.f, bj = 0.f;
        if (k > 0 && k < nt) {
            const float xi = (float)j / (float)(nxi - 1);
            const float wj = (j == 0 || j == nxi - 1) ? 0.5f : 1.f;
            const float qbar = scale * wj * dq[j];
            const float D = F[k] - F[k - 1];
            const float r = qbar * a.dt / (D * D);
            aj = r * (xi - F[k]);
            bj = -r * (xi - F[k - 1]);
        }
        A[j] = aj;
        Bq[j] = bj;
    }
    __syncthreads();
    block_scan<0, true>(A, nxi, red);
    block_scan<0, true>(Bq, nxi, red);
    // H_k into F (no longer needed), k = 0..nt-1
    for (int k = threadIdx.x; k < nt; k += NT_W2) {
        const int jk = lower_bound_i(ks, nxi, k);
        const int jk1 = lower_bound_i(ks, nxi, k + 1);
        F[k] = (jk1 < nxi ? A[jk1] : 0.f) + (jk < nxi ? Bq[jk] : 0.f);
    }
    __syncthreads();
    float zp = 0.f;
    for (int m = threadIdx.x; m < nt; m += NT_W2) {
        const float hm = m >= 1 ? F[m] : 0.f;
        const float hm1 = (m + 1 < nt) ? F[m + 1] : 0.f;
        const float pb = 0.5f * a.dt * (hm + hm1);
        Fm[m] = pb;
        zp += pb * y[m];
    }
    const float zsum = block_reduce<0, NT_W2>(zp, red);
    const float inv = 1.f / (Z + a.eps);
    const float zbar = -zsum * inv * inv;
    for (int m = threadIdx.x; m < nt; m += NT_W2) {
        const float wm = (m == 0 || m == nt - 1) ? 0.5f : 1.f;
        const float yb = Fm[m] * inv + zbar * a.dt * wm;
        ad[m] = om[m] * yb;
    }
}

W2Args make_w2(const Plan &pl, unsigned char *ctx)
{
    W2Args a;
    a.nt = pl.p.nt;
    a.nxi = pl.w2.n_xi;
    a.ntr = pl.p.ns * pl.p.nr;
    a.dt = pl.p.dt;
    a.k = pl.w2.k;
    a.cfac = pl.w2.cshift_factor;
    a.eps = pl.w2.eps_density;
    a.c = ctx_ptrs(pl, ctx);
    return a;
}

}  // namespace

size_t w2_trace_smem(int nt, int nxi) { return (3 * (size_t)nt + 4 * (size_t)nxi) * 4; }

cudaError_t launch_w2_prepare(const Plan &pl, const float *d_obs, unsigned char *ctx,
                              cudaStream_t st)
{
    W2Args a = make_w2(pl, ctx);
    const int B = pl.p.batch;
    k_obs_max<<<B, 1024, 0, st>>>(d_obs, (size_t)a.ntr * a.nt, a.c.M);
    const size_t sm = 3 * (size_t)a.nt * 4;
    cudaError_t e = cudaFuncSetAttribute(k_obs_trace, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_obs_trace<<<B * a.ntr, NT_W2, sm, st>>>(d_obs, a);
    k_sum_traces<<<B, NT_W2, 0, st>>>(a.c.s_tr, a.ntr, nullptr, a.c.S);
    return cudaGetLastError();
}

cudaError_t launch_w2_misfit(const Plan &pl, const unsigned char *ctx, const float *d_syn,
                             float *J, float *w2_out, float *adj, float *w2_scratch,
                             cudaStream_t st)
{
    W2Args a = make_w2(pl, const_cast<unsigned char *>(ctx));
    const int B = pl.p.batch;
    float *w2d = w2_out ? w2_out : w2_scratch;
    const size_t sm = w2_trace_smem(a.nt, a.nxi);
    cudaError_t e = cudaFuncSetAttribute(k_misfit_trace,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_misfit_trace<<<B * a.ntr, NT_W2, sm, st>>>(d_syn, a, w2d, adj);
    k_sum_traces<<<B, NT_W2, 0, st>>>(w2d, a.ntr, a.c.S, J);
    return cudaGetLastError();
}

}  // namespace fwi
