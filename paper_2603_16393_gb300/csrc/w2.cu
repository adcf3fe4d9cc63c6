// w2.cu -- weighted, normalised Wasserstein-2 misfit (Sec. 5.1, 6.2) and its
// exact derivative, one CTA per trace.
//
// Per trace (Sec. 6.2 numerics), written in the un-normalised running sum
//   G_0 = 0,  G_k = sum_{i=1..k} (y_{i-1} + y_i),   y = omega d + c'
// The trapezoid CDF is F_k = G_k / Gtot with Gtot = G_{nt-1} + 2 eps'/dt
// (because Z = dt G_{nt-1} / 2).  A synthetic trace can lie mostly below the
// shift taken from the observed data, so Gtot may be negative; with
// s = sign(Gtot) both sides of F_k >= xi_j are multiplied by s |Gtot| and the
// CDF is worked in the sign-corrected sums G~ = s G:
//   k*_j  = min{k : F_k >= xi_j} = min{k : G~_k >= t_j},  t_j = xi_j |Gtot|
//   Q_j   = t_{k*-1} + dt (t_j - G_{k*-1}) / (G_{k*} - G_{k*-1})   (clamped at the ends)
//   W2    = (dxi sum_j w_j (Q_j - Qobs_j)^2)^(1/2),  J = sum W2 / S_obs
// Quantiles are kept as (bracket base index, fraction in [0,1]); the
// difference of two quantiles is then an exact integer number of samples
// plus a difference of fractions, without cancellation.
//
// Reverse pass (no scatter).  With a_j, b_j the contributions of node j to
// dJ/dG_{k*-1} and dJ/dG_{k*}, c_j = dJ/dQ_j dt xi_j / D_j its contribution
// to dJ/dG_{nt-1} through t_j, and k*_j non-decreasing in j:
//   H_k = sum_{k' >= k} dJ/dG_{k'} = SA[J(k+1)] + SB[J(k)] + C [k <= nt-1],
// with SA, SB suffix sums over j, J(k) = min{j : k*_j >= k}, C = sum_j c_j;
//   dJ/dy_m = s (H_m [m >= 1] + H_{m+1}),   dJ/dd_m = omega_m dJ/dy_m,
// where H is taken with respect to G~ (the interpolation fraction is the
// same in G and G~, and t_j depends on G~_{nt-1} through xi_j).
//
// Precision: everything is float32; the running sums, the thresholds, the
// suffix sums and C are double-float (hi + lo float pairs, ~48-bit
// mantissa), because quantiles of two close distributions are compared and
// dJ/dy has the mean of dJ/dG removed (J is invariant to a rescaling of y).
// Every reduction has a fixed order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int NT_W2 = 256;          // threads per trace CTA
constexpr int NW_W2 = NT_W2 / 32;
constexpr unsigned FULL = 0xffffffffu;

// Shared-memory arrays of a trace are padded: element k of an 8-byte (df)
// array sits at pd(k), one gap every 16 elements, and of a 4-byte array at
// pw(k), one gap every 32.  A thread that owns a contiguous block of 4
// elements then meets the other threads of its half-warp (or warp) in
// distinct banks at every step of the block.
__device__ __forceinline__ int pd(int k) { return k + (k >> 4); }
__device__ __forceinline__ int pw(int k) { return k + (k >> 5); }
__host__ __device__ constexpr size_t pd_len(int n) { return (size_t)n + (n >> 4) + 1; }
__host__ __device__ constexpr size_t pw_len(int n) { return (size_t)n + (n >> 5) + 1; }
// Regions of the misfit kernel, each reused once its first array is dead:
//   R1: G (CDF build .. SA/SB terms), then H (suffix sums per sample)
//   R2: Gm (CDF build .. quantiles), then SA (terms and their suffix sums)
//   R3: y (CDF build), then SB
// plus dq and ks (quantiles .. reverse pass).
__host__ __device__ constexpr size_t max_len(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ constexpr size_t r2_len(int nt, int nxi)
{
    return max_len(pd_len(nt), pd_len(nxi));
}
__host__ __device__ constexpr size_t r3_len(int nt, int nxi)
{
    return max_len(pd_len(nxi), (size_t)(nt + 1) / 2);
}

// ---------------------------------------------------------------- double-float
// A value hi + lo with |lo| <= ulp(hi)/2 (Knuth two-sum / Dekker two-product,
// error-free transformations in float32).
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_div_f(df a, float b)
{
    const float q1 = __fdiv_rn(a.hi, b);
    const df p = {__fmul_rn(q1, b), __fmaf_rn(q1, b, -__fmul_rn(q1, b))};
    const df r = df_sub(a, p);
    const float q2 = __fdiv_rn(r.hi, b);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ bool df_lt(df a, df b)
{
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ df df_max(df a, df b) { return df_lt(a, b) ? b : a; }
__device__ __forceinline__ df df_shfl_up(df v, int o)
{
    return {__shfl_up_sync(FULL, v.hi, o), __shfl_up_sync(FULL, v.lo, o)};
}
__device__ __forceinline__ df df_shfl_xor(df v, int o)
{
    return {__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
}

// ---------------------------------------------------------------- block helpers
// OP: 0 sum, 1 max, 2 min.
template <int OP>
__device__ __forceinline__ float fcomb(float a, float b)
{
    return OP == 0 ? a + b : OP == 1 ? fmaxf(a, b) : fminf(a, b);
}
template <int OP>
__device__ __forceinline__ float fident()
{
    return OP == 0 ? 0.f : OP == 1 ? -INFINITY : INFINITY;
}
template <int OP>
__device__ __forceinline__ df dcomb(df a, df b)
{
    return OP == 0 ? df_add(a, b) : df_max(a, b);
}
template <int OP>
__device__ __forceinline__ df dident()
{
    return OP == 0 ? df{0.f, 0.f} : df{-INFINITY, 0.f};
}

// float reduction over the block; red holds NTH/32 + 1 floats
template <int OP, int NTH>
__device__ float block_reduce(float v, float *red)
{
    constexpr int NW = NTH / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fcomb<OP>(v, __shfl_xor_sync(FULL, v, o));
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float u = lane < NW ? red[lane] : fident<OP>();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u = fcomb<OP>(u, __shfl_xor_sync(FULL, u, o));
        if (lane == 0) red[NW] = u;
    }
    __syncthreads();
    return red[NW];
}

// double-float sum over the block; red holds NW_W2 + 1 df
__device__ df block_sum_df(df v, df *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        df u = lane < NW_W2 ? red[lane] : df{0.f, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u = df_add(u, df_shfl_xor(u, o));
        if (lane == 0) red[NW_W2] = u;
    }
    __syncthreads();
    return red[NW_W2];
}

// In-place inclusive double-float scan (OP 0: sum, 1: max) of arr[0..n) in
// shared memory (padded, pd), blocked arrangement; REV scans from the end
// (suffix scan).
template <int OP, bool REV>
__device__ void block_scan_df(df *arr, int n, df *red)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int per = (n + NT_W2 - 1) / NT_W2;
    const int lo = tid * per, hi = min(lo + per, n);
    df run = dident<OP>();
    for (int i = lo; i < hi; ++i) {
        const int k = REV ? n - 1 - i : i;
        run = dcomb<OP>(run, arr[pd(k)]);
        arr[pd(k)] = run;
    }
    df incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const df y = df_shfl_up(incl, o);
        if (lane >= o) incl = dcomb<OP>(y, incl);
    }
    __syncthreads();
    if (lane == 31) red[w] = incl;
    __syncthreads();
    if (w == 0) {
        df u = lane < NW_W2 ? red[lane] : dident<OP>();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const df y = df_shfl_up(u, o);
            if (lane >= o) u = dcomb<OP>(y, u);
        }
        if (lane < NW_W2) red[lane] = u;
    }
    __syncthreads();
    const df prev = df_shfl_up(incl, 1);
    df off = lane > 0 ? prev : dident<OP>();
    if (w > 0) off = lane > 0 ? dcomb<OP>(red[w - 1], off) : red[w - 1];
    if (tid > 0) {
        for (int i = lo; i < hi; ++i) {
            const int k = REV ? n - 1 - i : i;
            arr[pd(k)] = dcomb<OP>(off, arr[pd(k)]);
        }
    }
    __syncthreads();
}

// first k in [0, n) with a[k] >= x (a non-decreasing, padded); n if none
__device__ __forceinline__ int lower_bound_df(const df *a, int n, df x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (df_lt(a[pd(mid)], x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound_i(const int *a, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[pw(mid)] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The same first index with a[i] >= x, given that every a[i] < x for i < k
// (a nondecreasing, x no smaller than at an earlier search that returned k):
// a few steps forward from k, then a binary search of what is left.  The
// threads of a trace take contiguous blocks of increasing x, so a thread
// searches once in full and then mostly steps.
constexpr int kWalk = 8;
__device__ __forceinline__ int lower_bound_df_from(const df *a, int n, df x, int k)
{
    for (int s = 0; s < kWalk && k < n; ++s, ++k)
        if (!df_lt(a[pd(k)], x)) return k;
    int lo = k, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (df_lt(a[pd(mid)], x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound_i_from(const int *a, int n, int x, int k)
{
    for (int s = 0; s < kWalk && k < n; ++s, ++k)
        if (a[pw(k)] >= x) return k;
    int lo = k, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[pw(mid)] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct CtxPtrs {
    float *M;        // [B]
    float *S;        // [B] sum of s_tr (Eq. final_objective denominator)
    float *S2;       // [B] sum of s_tr^2 (the squared raw objective's denominator)
    float *cshift;   // [B][ntr]
    float *s_tr;     // [B][ntr]
    float *omega;    // [B][ntr][nt]
    int *Qb;         // [B][ntr][nxi] bracket base index of the observed quantile
    float *Qf;       // [B][ntr][nxi] fraction inside the bracket
};

inline CtxPtrs ctx_ptrs(const Plan &pl, unsigned char *ctx)
{
    CtxPtrs c;
    c.M = (float *)(ctx + pl.ctx_M);
    c.S = (float *)(ctx + pl.ctx_S);
    c.S2 = (float *)(ctx + pl.ctx_S2);
    c.cshift = (float *)(ctx + pl.ctx_cshift);
    c.s_tr = (float *)(ctx + pl.ctx_str);
    c.omega = (float *)(ctx + pl.ctx_omega);
    c.Qb = (int *)(ctx + pl.ctx_Qb);
    c.Qf = (float *)(ctx + pl.ctx_Qf);
    return c;
}

struct W2Args {
    int nt, nxi, ntr;           // ntr = ns * nr traces per instance
    float dt, k, cfac, eps2dt;  // eps2dt = 2 eps' / dt
    int squared;                // J = sum W2^2 / S2 instead of sum W2 / S
    CtxPtrs c;
};

// y = omega d + c' with both roundings explicit, so that the observation
// preparation and the misfit map identical data to identical densities.
__device__ __forceinline__ float shifted(float w, float d, float cs)
{
    return __fadd_rn(__fmul_rn(w, d), cs);
}

// Sign-corrected running sums G~ = s G and their running max Gm from y (all
// in shared memory); returns the quantile step unit = |Gtot| / (nxi - 1) and
// writes s = sign(Gtot) (+1 when Gtot is zero).
__device__ df build_cdf(const float *y, df *G, df *Gm, int nt, int nxi, float eps2dt, df *red,
                        float *sgn)
{
    for (int i = threadIdx.x; i < nt; i += NT_W2)
        G[pd(i)] = i == 0 ? df{0.f, 0.f} : two_sum(y[i - 1], y[i]);
    __syncthreads();
    block_scan_df<0, false>(G, nt, red);
    df gtot = df_add(G[pd(nt - 1)], df_from(eps2dt));
    const bool neg = gtot.hi < 0.f;
    __syncthreads();                  // every thread has read G[nt - 1]
    for (int i = threadIdx.x; i < nt; i += NT_W2) {
        const df g = neg ? df_neg(G[pd(i)]) : G[pd(i)];
        G[pd(i)] = g;
        Gm[pd(i)] = g;
    }
    __syncthreads();
    block_scan_df<1, false>(Gm, nt, red);
    if (neg) gtot = df_neg(gtot);
    *sgn = neg ? -1.f : 1.f;
    return df_div_f(gtot, (float)(nxi - 1));
}

// Quantile of node j as (base, frac): Q = (base + frac) dt.  Writes k*.
// Contiguous block [*i0, *i1) of 0..n-1 for this thread of an NT_W2 block.
__device__ __forceinline__ void thread_block(int n, int *i0, int *i1)
{
    const int c = (n + NT_W2 - 1) / NT_W2;
    *i0 = min(n, (int)threadIdx.x * c);
    *i1 = min(n, *i0 + c);
}

// Quantile node j of the CDF G (running maximum Gm) by the generalised
// inverse: bracket k = first index with Gm[k] >= t_j = unit j; kfrom = k of
// an earlier node of this thread (or 0: full search).
__device__ __forceinline__ void quantile(const df *G, const df *Gm, int nt, df unit, int j,
                                         int kfrom, int *kst, int *base, float *frac, df *tj)
{
    const df t = df_mul_f(unit, (float)j);
    const int k = kfrom > 0 ? lower_bound_df_from(Gm, nt, t, kfrom) : lower_bound_df(Gm, nt, t);
    *kst = k;
    *tj = t;
    if (k == 0) { *base = 0; *frac = 0.f; return; }
    if (k == nt) { *base = nt - 1; *frac = 0.f; return; }
    *base = k - 1;
    *frac = __fdiv_rn(df_f(df_sub(t, G[pd(k - 1)])), df_f(df_sub(G[pd(k)], G[pd(k - 1)])));
}

// ------------------------------------------------------------------ kernels
// M[b] = max |d_obs| of instance b (blockIdx.y) over its slices (blockIdx.x):
// each CTA reduces one slice and folds it in with an integer atomicMax on the
// float bits (M zeroed first; |d| >= 0, whose bit patterns order as the
// values do, so the result does not depend on the order of the CTAs).
constexpr int kObsMaxThreads = 256;
__global__ void __launch_bounds__(kObsMaxThreads)
    k_obs_max(const float *__restrict__ d, size_t per_inst, size_t slice, float *__restrict__ M)
{
    __shared__ float red[kObsMaxThreads / 32 + 1];
    const float *db = d + (size_t)blockIdx.y * per_inst;
    const size_t i0 = (size_t)blockIdx.x * slice;
    const size_t i1 = i0 + slice < per_inst ? i0 + slice : per_inst;
    float m = 0.f;
    for (size_t i = i0 + threadIdx.x; i < i1; i += kObsMaxThreads) m = fmaxf(m, fabsf(db[i]));
    m = block_reduce<1, kObsMaxThreads>(m, red);
    if (threadIdx.x == 0)
        atomicMax(reinterpret_cast<unsigned *>(M) + blockIdx.y, __float_as_uint(m));
}

__global__ void __launch_bounds__(NT_W2) k_obs_trace(const float *__restrict__ d_obs, W2Args a)
{
    extern __shared__ df smd[];
    __shared__ df red[NW_W2 + 2];
    __shared__ float redf[NW_W2 + 2];
    const int tr_g = blockIdx.x;                 // b * ntr + tr
    const int b = tr_g / a.ntr;
    df *G = smd, *Gm = G + pd_len(a.nt);
    float *y = (float *)(Gm + pd_len(a.nt));
    const float *d = d_obs + (size_t)tr_g * a.nt;
    float *om = a.c.omega + (size_t)tr_g * a.nt;
    const float M = a.c.M[b];
    float mn = INFINITY;
    for (int i = threadIdx.x; i < a.nt; i += NT_W2) {
        const float di = d[i];
        const float w = 1.f / (1.f + a.k * (M > 0.f ? fabsf(di) / M : 0.f));
        om[i] = w;
        mn = fminf(mn, __fmul_rn(w, di));
    }
    mn = block_reduce<2, NT_W2>(mn, redf);
    const float cs = a.cfac * fabsf(mn);
    if (threadIdx.x == 0) a.c.cshift[tr_g] = cs;
    for (int i = threadIdx.x; i < a.nt; i += NT_W2) y[i] = shifted(om[i], d[i], cs);
    __syncthreads();
    float sgn;
    const df unit = build_cdf(y, G, Gm, a.nt, a.nxi, a.eps2dt, red, &sgn);
    int *Qb = a.c.Qb + (size_t)tr_g * a.nxi;
    float *Qf = a.c.Qf + (size_t)tr_g * a.nxi;
    float part = 0.f;
    int j0, j1, kprev = 0;
    thread_block(a.nxi, &j0, &j1);
    for (int j = j0; j < j1; ++j) {
        int k, base;
        float frac;
        df t;
        quantile(G, Gm, a.nt, unit, j, kprev, &k, &base, &frac, &t);
        kprev = k;
        Qb[j] = base;
        Qf[j] = frac;
        const float q = ((float)base + frac) * a.dt;
        const float wj = (j == 0 || j == a.nxi - 1) ? 0.5f : 1.f;
        part += wj * q * q;
    }
    const float s2 = block_reduce<0, NT_W2>(part, redf);
    if (threadIdx.x == 0) a.c.s_tr[tr_g] = sqrtf(s2 / (float)(a.nxi - 1));
}

// out[b] = sum_i v[b][i] (SQ: v^2; fixed order), divided by div[b] if given
template <bool SQ>
__global__ void __launch_bounds__(NT_W2) k_sum_traces(const float *__restrict__ v, int ntr,
                                                      const float *__restrict__ div,
                                                      float *__restrict__ out)
{
    __shared__ float red[NW_W2 + 2];
    const float *vb = v + (size_t)blockIdx.x * ntr;
    float part = 0.f;
    for (int i = threadIdx.x; i < ntr; i += NT_W2) part += SQ ? vb[i] * vb[i] : vb[i];
    const float s = block_reduce<0, NT_W2>(part, red);
    if (threadIdx.x == 0) out[blockIdx.x] = div ? s / div[blockIdx.x] : s;
}

// six traces a SM: 40 registers a thread (x 256 threads x 6 = 61 440) and
// 33.8 KB of shared arrays a trace at 1000 samples and nodes
__global__ void __launch_bounds__(NT_W2, 6)
    k_misfit_trace(const float *__restrict__ d_syn, W2Args a, float *__restrict__ w2_dst,
                   float *__restrict__ adj)
{
    extern __shared__ df smd[];
    __shared__ df red[NW_W2 + 2];
    __shared__ float redf[NW_W2 + 2];
    const int tr_g = blockIdx.x;
    const int b = tr_g / a.ntr;
    const int nt = a.nt, nxi = a.nxi;
    df *G = smd, *Gm = G + pd_len(nt), *SB = Gm + r2_len(nt, nxi);
    df *SA = Gm, *H = G;
    float *y = (float *)SB;
    float *dq = (float *)(SB + r3_len(nt, nxi));
    int *ks = (int *)(dq + pw_len(nxi));
    const float *d = d_syn + (size_t)tr_g * nt;
    const float *om = a.c.omega + (size_t)tr_g * nt;
    const float cs = a.c.cshift[tr_g];
    for (int i = threadIdx.x; i < nt; i += NT_W2) y[i] = shifted(om[i], d[i], cs);
    __syncthreads();
    float sgn;
    const df unit = build_cdf(y, G, Gm, nt, nxi, a.eps2dt, red, &sgn);
    const int *Qb = a.c.Qb + (size_t)tr_g * nxi;
    const float *Qf = a.c.Qf + (size_t)tr_g * nxi;
    float part = 0.f;
    int j0, j1, kprev = 0;
    thread_block(nxi, &j0, &j1);
    for (int j = j0; j < j1; ++j) {
        int k, base;
        float frac;
        df t;
        quantile(G, Gm, nt, unit, j, kprev, &k, &base, &frac, &t);
        kprev = k;
        // (base - base_obs) is exact; the fractions are in [0, 1]
        const float diff = ((float)(base - Qb[j]) + (frac - Qf[j])) * a.dt;
        dq[pw(j)] = diff;
        ks[pw(j)] = k;
        const float wj = (j == 0 || j == nxi - 1) ? 0.5f : 1.f;
        part += wj * diff * diff;
    }
    const float dxi = 1.f / (float)(nxi - 1);
    const float W2sq = dxi * block_reduce<0, NT_W2>(part, redf);
    const float W2 = sqrtf(W2sq);
    if (threadIdx.x == 0) w2_dst[tr_g] = a.squared ? W2sq : W2;
    if (!adj) return;
    float *ad = adj + (size_t)tr_g * nt;
    if (W2 == 0.f) {   // W2 (non-differentiable there) or W2^2 (derivative 0): zero
        for (int i = threadIdx.x; i < nt; i += NT_W2) ad[i] = 0.f;
        return;
    }
    // dJ/dQ_j = scale w_j (Q_j - Qobs_j)
    const float scale = a.squared ? 2.f * dxi / a.c.S2[b] : dxi / (W2 * a.c.S[b]);
    df cpart = {0.f, 0.f};
    for (int j = threadIdx.x; j < nxi; j += NT_W2) {
        const int k = ks[pw(j)];
        df aj = {0.f, 0.f}, bj = {0.f, 0.f};
        if (k > 0 && k < nt) {
            const df t = df_mul_f(unit, (float)j);
            const float wj = (j == 0 || j == nxi - 1) ? 0.5f : 1.f;
            const float qbar = scale * wj * dq[pw(j)];        // dJ/dQ_j
            const float D = df_f(df_sub(G[pd(k)], G[pd(k - 1)]));
            const float r = qbar * a.dt / (D * D);
            aj = df_from(r * df_f(df_sub(t, G[pd(k)])));      // -> dJ/dG_{k-1}
            bj = df_from(-r * df_f(df_sub(t, G[pd(k - 1)]))); // -> dJ/dG_k
            // through t_j = xi_j Gtot -> dJ/dG_{nt-1}
            cpart = df_add(cpart, df_from(qbar * a.dt * ((float)j * dxi) / D));
        }
        SA[pd(j)] = aj;
        SB[pd(j)] = bj;
    }
    const df C = block_sum_df(cpart, red);
    block_scan_df<0, true>(SA, nxi, red);
    block_scan_df<0, true>(SB, nxi, red);
    // H_k into G's region (no longer needed), k = 0..nt-1 (H_nt = 0); j(k) = first
    // node whose bracket is >= k grows with k: a block of k per thread
    int k0, k1;
    thread_block(nt, &k0, &k1);
    if (k0 < k1) {
        int jk = lower_bound_i(ks, nxi, k0);
        for (int k = k0; k < k1; ++k) {
            const int jk1 = lower_bound_i_from(ks, nxi, k + 1, jk);
            df h = C;
            if (jk1 < nxi) h = df_add(h, SA[pd(jk1)]);
            if (jk < nxi) h = df_add(h, SB[pd(jk)]);
            H[pd(k)] = h;
            jk = jk1;
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < nt; m += NT_W2) {
        df yb = m + 1 < nt ? H[pd(m + 1)] : df{0.f, 0.f};
        if (m >= 1) yb = df_add(yb, H[pd(m)]);
        ad[m] = om[m] * (sgn * df_f(yb));
    }
}

W2Args make_w2(const Plan &pl, unsigned char *ctx)
{
    W2Args a;
    a.nt = pl.p.nt;
    a.nxi = pl.w2.n_xi;
    a.ntr = pl.p.ns * pl.p.nr;
    a.dt = (float)pl.p.dt;
    a.k = (float)pl.w2.k;
    a.cfac = (float)pl.w2.cshift_factor;
    a.eps2dt = (float)(2.0 * (double)pl.w2.eps_density / (double)pl.p.dt);
    a.squared = pl.w2.squared;
    a.c = ctx_ptrs(pl, ctx);
    return a;
}

size_t obs_trace_smem(int nt) { return 2 * pd_len(nt) * sizeof(df) + (size_t)nt * 4; }

}  // namespace

size_t w2_trace_smem(int nt, int nxi)
{
    // G then H; Gm then SA; y then SB; dq, ks
    return (pd_len(nt) + r2_len(nt, nxi) + r3_len(nt, nxi)) * sizeof(df) + 2 * pw_len(nxi) * 4;
}

cudaError_t launch_w2_prepare(const Plan &pl, const float *d_obs, unsigned char *ctx,
                              cudaStream_t st)
{
    W2Args a = make_w2(pl, ctx);
    const int B = pl.p.batch;
    {
        // about eight CTAs per SM over all instances, slices of >= 4096 samples
        const size_t per_inst = (size_t)a.ntr * a.nt;
        size_t nsl = (per_inst + 4095) / 4096;
        const size_t cap = (size_t)(B < 1216 ? 1216 / B : 1);
        if (nsl > cap) nsl = cap;
        if (nsl < 1) nsl = 1;
        const size_t slice = (per_inst + nsl - 1) / nsl;
        cudaError_t e0 = cudaMemsetAsync(a.c.M, 0, (size_t)B * sizeof(float), st);
        if (e0 != cudaSuccess) return e0;
        k_obs_max<<<dim3((unsigned)nsl, (unsigned)B), kObsMaxThreads, 0, st>>>(d_obs, per_inst,
                                                                             slice, a.c.M);
    }
    const size_t sm = obs_trace_smem(a.nt);
    cudaError_t e = cudaFuncSetAttribute(k_obs_trace, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_obs_trace<<<B * a.ntr, NT_W2, sm, st>>>(d_obs, a);
    k_sum_traces<false><<<B, NT_W2, 0, st>>>(a.c.s_tr, a.ntr, nullptr, a.c.S);
    k_sum_traces<true><<<B, NT_W2, 0, st>>>(a.c.s_tr, a.ntr, nullptr, a.c.S2);
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
    k_sum_traces<false><<<B, NT_W2, 0, st>>>(w2d, a.ntr, a.squared ? a.c.S2 : a.c.S, J);
    return cudaGetLastError();
}

}  // namespace fwi
