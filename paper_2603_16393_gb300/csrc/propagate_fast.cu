// propagate_fast.cu -- shared-memory-resident propagators with a compile-time
// shared-memory pitch (every stencil offset is an immediate) and fixed
// 22-row column strips, for padded grids that fit one CTA.
//
// Forward (Eq. 1, Sec. 2.1 / 6.1), written in increment form: with
// v^{j+1/2} = u^{j+1} - u^j the damped leapfrog
//   u^{j+1} = A (2 u^j - B u^{j-1} + kappa (L u^j + s^j))
// is exactly
//   v^{j+1/2} = A B v^{j-1/2} + kappa A (L u^j + s^j),   u^{j+1} = u^j + v^{j+1/2}.
// Carrying the small increment instead of u^{j-1} keeps float32 round-off
// from growing with the nearly double root of the recurrence at low
// frequency; the Laplacian is evaluated on neighbour differences
// ((u_{k-1} - u_k) + (u_{k+1} - u_k)) for the same reason.  The record of step
// j is L u^j (the point source is added back by the adjoint).
//
// Adjoint: psi^{j+1} = A (2 psi^j - B psi^{j-1} + kappa (L^T psi^j + R^T r^{nt-1-j}))
// (the discrete adjoint in the self-adjoint phi = kappa A mu form, reversed
// time), dJ/dv_pad = (2/v_pad) sum_j psi^{j+1} t^{nt-1-j}.  A receiver's
// adjoint source is folded into the owner-only old level,
// psi^{j-1} -= (kappa/B) q, which the update turns into + A kappa q.
//
// Shared memory: two time levels of the field with a two-cell ghost ring,
// pitch P (and, for the adjoint, kappa A per cell), plus a staging buffer for
// receiver samples.  Thread (x, strip) owns rows [22 strip, 22 strip + 22) at
// padded column x.  Rows past the padded grid are dead rows: kappa = 0 keeps
// them at zero, and they act as the zero ghosts below the grid.
#include <cuda_runtime.h>

#include <cmath>

#include "f32x2.cuh"
#include "fwi_device.cuh"
#include "fwi_internal.cuh"
#include "stencil_pair.cuh"
#include "tmem.cuh"

namespace fwi {

namespace {

constexpr int ROWS = kFastRows;

using dev::e_cell;
using dev::ex_of;
using dev::ez_of;
using dev::kappaA_cell;
using dev::ricker_scaled;

// ------------------------------------------------------------------ forward
template <int P, int PR, int TOPBC, bool STORE>
__device__ __forceinline__ void fwd_rows(const float *__restrict__ cp, float *__restrict__ np,
                                         const float *__restrict__ abp, float *__restrict__ sw,
                                         int NX, bool top_strip, float (&ka)[ROWS],
                                         float (&vi)[ROWS], const PropArgs &a)
{
    float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
    float Dp = w0 - wm1;      // u_z - u_{z-1}
    float Em2 = w0 - wm2;     // u_z - u_{z-2}      (E of row z-2)
    float Em1 = wp1 - wm1;    // u_{z+1} - u_{z-1}  (E of row z-1)
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const float *c = cp + r * P;
        const float wp2 = c[2 * P];
        const float Dn = wp1 - w0;
        const float E0 = wp2 - w0;
        const float dzA = Dn - Dp;                        // (u_{z-1}-u_z) + (u_{z+1}-u_z)
        const float dzB = E0 - Em2;                       // (u_{z-2}-u_z) + (u_{z+2}-u_z)
        const float dxA = (c[-1] - w0) + (c[1] - w0);
        const float dxB = (c[-2] - w0) + (c[2] - w0);
        float lap = a.cx1 * dxA;
        lap = fmaf(a.cx2, dxB, lap);
        lap = fmaf(a.cz1, dzA, lap);
        lap = fmaf(a.cz2, dzB, lap);
        vi[r] = fmaf(ka[r], lap, abp[r * P] * vi[r]);
        const float un = w0 + vi[r];
        np[r * P] = un;
        if (TOPBC == 1 && (r == 1 || r == 2)) {
            if (top_strip) np[-r * P] = un;               // mirrored ghost rows -1, -2
        }
        if (STORE) sw[r * PR] = lap;
        Dp = Dn;
        Em2 = Em1;
        Em1 = E0;
        wm2 = wm1;
        wm1 = w0;
        w0 = wp1;
        wp1 = wp2;
    }
}

template <int P, int PR, int NZM, int TOPBC, bool STORE>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1) k_fwd_fast(const __grid_constant__ PropArgs a)
{
    extern __shared__ float sm[];
    constexpr int FSZ = (NZM + 4) * P;
    float *U0 = sm, *U1 = sm + FSZ, *ABt = sm + 2 * FSZ, *ST = ABt + NZM * P;
    const int NX = a.NX, NZ = a.NZ;
    const int bs = blockIdx.x, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < 2 * FSZ; i += nth) sm[i] = 0.f;
    // A B = (1 - e)/(1 + e) per cell (e = eta dt / 2)
    for (int i = tid; i < NZM * P; i += nth) {
        const int pz = i / P, px = i - (i / P) * P;
        const double e = e_cell(px, pz, a);
        ABt[i] = (float)((1.0 - e) / (1.0 + e));
    }

    const int x = tid % NX, strip = tid / NX;
    const bool active = strip < a.nstrip;
    const int z0 = strip * ROWS;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    const int ixc = min(max(x - a.nb, 0), a.nx - 1);
    const float ex = ex_of(x, a);
    float ka[ROWS], vi[ROWS];
    int bad = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int z = z0 + r;
        float k = 0.f;
        if (active && z < NZ) {
            const float vv = vb[min(z, a.nz - 1) * a.nx + ixc];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, x, z, a);
        }
        ka[r] = k;
        vi[r] = 0.f;
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
        return;
    }
    const bool top_strip = active && z0 == 0;

    // source owner
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const int src_row = (active && x == sx && sz >= z0 && sz < z0 + ROWS) ? sz - z0 : -1;
    float ka_src = 0.f;
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
        if (r == src_row) ka_src = ka[r];

    const size_t plane = (size_t)a.nzs * PR;   // record planes use the pitch PR
    float *snap_bs = STORE ? a.snap + (size_t)bs * a.rec_planes * plane : nullptr;
    const int jb = a.j_begin;
    if (a.resume) {
        // state at step jb: field u^jb (a flat copy, with the mirrored ghost
        // rows -1, -2) and the owner's increments v^(jb-1/2)
        const size_t cells = (size_t)NZ * NX;
        const float *st = a.resume + (size_t)bs * 2 * cells;
        float *cur = (jb & 1) ? U1 : U0;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            const float u = st[i];
            cur[(z + 2) * P + xx + 2] = u;
            if (TOPBC == 1 && (z == 1 || z == 2)) cur[(2 - z) * P + xx + 2] = u;
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int z = z0 + r;
                if (z < NZ) vi[r] = st[cells + z * NX + x];
            }
        }
        __syncthreads();
    }

    for (int j0 = jb, nch = 0; j0 < a.j_end; j0 += nch) {
        nch = min(a.chunk, a.j_end - j0);
        if (a.ckpt) {
            // chunks end at checkpoint steps; the state at the first step of
            // a chunk that is one is saved here
            nch = min(nch, (j0 / a.ckpt_every + 1) * a.ckpt_every - j0);
            if (j0 % a.ckpt_every == 0) {
                const float *cur = (j0 & 1) ? U1 : U0;
                const size_t cl = (size_t)NZ * NX;
                float *st = a.ckpt + ((size_t)(j0 / a.ckpt_every) * gridDim.x + bs) * 2 * cl;
                for (int i = tid; i < NZ * NX; i += nth) {
                    const int z = i / NX, xx = i - (i / NX) * NX;
                    st[i] = cur[(z + 2) * P + xx + 2];
                }
                if (active) {
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        const int z = z0 + r;
                        if (z < NZ) st[cl + z * NX + x] = vi[r];
                    }
                }
            }
        }
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (active) {
                const float *cp = cur + (z0 + 2) * P + x + 2;
                float *np = nxt + (z0 + 2) * P + x + 2;
                float *sw = STORE ? snap_bs + (size_t)(j - a.rec_base) * plane + z0 * PR + x
                                  : nullptr;
                fwd_rows<P, PR, TOPBC, STORE>(cp, np, ABt + z0 * P + x, sw, NX, top_strip, ka, vi, a);
                if (src_row >= 0) {
                    // point source: + kappa A s at the source cell (increment and field)
                    const float d = ka_src * ricker_scaled(j, a);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r)
                        if (r == src_row) vi[r] += d;
                    np[src_row * P] += d;
                    if (TOPBC == 1 && top_strip && (src_row == 1 || src_row == 2))
                        np[-src_row * P] += d;
                }
            }
            __syncthreads();
            if (tid < a.nr) ST[jj * a.nr + tid] = nxt[(a.rec_pz[tid] + 2) * P + a.rec_px[tid] + 2];
        }
        __syncthreads();
        if (a.d_syn) {
            float *db = a.d_syn + (size_t)bs * a.nr * a.nt;
            for (int e = tid; e < nch * a.nr; e += nth) {
                const int i = e / nch, jj = e - (e / nch) * nch;
                db[(size_t)i * a.nt + j0 + jj] = ST[jj * a.nr + i];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ forward, column pairs
// Same arithmetic as k_fwd_fast, but each thread owns two adjacent columns
// (x, x+1) and 11 rows, and moves them as float2: per row three 8-byte
// loads ((x-2, x-1), the window row z+2, (x+2, x+3)) and one 8-byte store
// serve two cell-updates.  The two columns go through the packed f32x2
// instructions (one instruction per operation for both cells; results
// bitwise those of the scalar code).  Needs an even padded width.
constexpr int ROWS2 = kFastRows / 2;

// One (model, shot) unit bs of a plan: the whole forward time loop of the
// column-pair kernel (k_fwd_pair runs one unit a CTA, k_fwd_pair_queue draws
// units of several plans from a counter)
template <int P, int PR, int NZM, int TOPBC, bool STORE, bool AHEAD>
__device__ __forceinline__ void fwd_pair_unit(const PropArgs &a, const PropArgs &c, const int bs)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int FSZ = (NZM + 4) * P;
    float *U0 = sm, *U1 = sm + FSZ, *ABt = sm + 2 * FSZ, *ST = ABt + NZM * P;
    const int NX = a.NX, NZ = a.NZ;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < 2 * FSZ; i += nth) sm[i] = 0.f;
    for (int i = tid; i < NZM * P; i += nth) {
        const int pz = i / P, px = i - (i / P) * P;
        const double e = e_cell(px, pz, a);
        ABt[i] = (float)((1.0 - e) / (1.0 + e));
    }

    const int NXP = NX / 2;
    const int xp = tid % NXP, strip = tid / NXP;
    const bool active = strip < a.nstrip;
    const int x = 2 * xp, z0 = strip * ROWS2;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    float2 ka[ROWS2], vi[ROWS2];
    int bad = 0;
#pragma unroll
    for (int r = 0; r < ROWS2; ++r) {
        float k[2] = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int z = z0 + r;
            if (active && z < NZ) {
                const int ixc = min(max(x + c - a.nb, 0), a.nx - 1);
                const float vv = vb[min(z, a.nz - 1) * a.nx + ixc];
                if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
                k[c] = kappaA_cell(vv, x + c, z, a);
            }
        }
        ka[r] = make_float2(k[0], k[1]);
        vi[r] = make_float2(0.f, 0.f);
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
        return;
    }
    const bool top_strip = active && z0 == 0;

    // source owner: row and column inside this thread's 11 x 2 block
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const int src_k = (active && (sx >> 1) == xp && sz >= z0 && sz < z0 + ROWS2)
                          ? 2 * (sz - z0) + (sx & 1) : -1;
    const int jb = a.j_begin;
    // record plane of the current step (advanced by one plane per step)
    float *sw = STORE ? a.snap + ((size_t)bs * a.rec_planes + (jb - a.rec_base)) * a.nzs * PR +
                            z0 * PR + x
                      : nullptr;
    if (a.resume) {
        // state at step jb: field u^jb and increment v^(jb-1/2)
        const size_t cells = (size_t)NZ * NX;
        const float *st = a.resume + (size_t)bs * 2 * cells;
        float *cur = (jb & 1) ? U1 : U0;
        for (int i = tid; i < NZ * NX; i += nth) {   // flat copy of u^jb
            const int z = i / NX, xx = i - (i / NX) * NX;
            const float u = st[i];
            cur[(z + 2) * P + xx + 2] = u;
            if (TOPBC == 1 && (z == 1 || z == 2)) cur[(2 - z) * P + xx + 2] = u;
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < ROWS2; ++r) {
                const int z = z0 + r;
                if (z < NZ) vi[r] = *(const float2 *)(st + cells + z * NX + x);
            }
        }
        __syncthreads();
    }

    for (int j0 = jb, nch = 0; j0 < a.j_end; j0 += nch) {
        nch = min(a.chunk, a.j_end - j0);
        if (a.ckpt) {
            // chunks end at checkpoint steps; the state at the first step of
            // a chunk that is one is saved here
            nch = min(nch, (j0 / a.ckpt_every + 1) * a.ckpt_every - j0);
            if (j0 % a.ckpt_every == 0) {
                const float *cur = (j0 & 1) ? U1 : U0;
                const size_t cl = (size_t)NZ * NX;
                float *st = a.ckpt + ((size_t)(j0 / a.ckpt_every) * a.units + bs) * 2 * cl;
                for (int i = tid; i < NZ * NX; i += nth) {
                    const int z = i / NX, xx = i - (i / NX) * NX;
                    st[i] = cur[(z + 2) * P + xx + 2];
                }
                if (active) {
#pragma unroll
                    for (int r = 0; r < ROWS2; ++r) {
                        const int z = z0 + r;
                        if (z < NZ) *(float2 *)(st + cl + z * NX + x) = vi[r];
                    }
                }
            }
        }
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (active) {
                const float *cp = cur + (z0 + 2) * P + x + 2;
                float *np = nxt + (z0 + 2) * P + x + 2;
                fwd_rows_pair<P, PR, ROWS2, TOPBC, STORE, AHEAD>(cp, np, ABt + z0 * P + x, sw,
                                                                 top_strip, ka, vi, c);
                if (src_k >= 0) {
                    // point source: + kappa A s at the source cell (increment and field)
                    float kas = 0.f;
#pragma unroll
                    for (int k = 0; k < ROWS2; ++k) {
                        if (2 * k == src_k) kas = ka[k].x;
                        if (2 * k + 1 == src_k) kas = ka[k].y;
                    }
                    const float d = kas * ricker_scaled(j, c);
#pragma unroll
                    for (int k = 0; k < ROWS2; ++k) {
                        if (2 * k == src_k) vi[k].x += d;
                        if (2 * k + 1 == src_k) vi[k].y += d;
                    }
                    const int sz = a.src_pz[s], sx = a.src_px[s];
                    nxt[(sz + 2) * P + sx + 2] += d;
                    if (TOPBC == 1 && (sz == 1 || sz == 2)) nxt[(2 - sz) * P + sx + 2] += d;
                }
            }
            if (STORE) sw += (size_t)a.nzs * PR;
            __syncthreads();
            if (tid < a.nr) ST[jj * a.nr + tid] = nxt[(a.rec_pz[tid] + 2) * P + a.rec_px[tid] + 2];
        }
        __syncthreads();
        if (a.d_syn) {
            float *db = a.d_syn + (size_t)bs * a.nr * a.nt;
            for (int e = tid; e < nch * a.nr; e += nth) {
                const int i = e / nch, jj = e - (e / nch) * nch;
                db[(size_t)i * a.nt + j0 + jj] = ST[jj * a.nr + i];
            }
        }
        __syncthreads();
    }
}

template <int P, int PR, int NZM, int TOPBC, bool STORE>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1)
k_fwd_pair(const __grid_constant__ PropArgs a)
{
    fwd_pair_unit<P, PR, NZM, TOPBC, STORE, true>(a, a, blockIdx.x);
}

// Persistent: every CTA draws units (plan p, unit bs) from the counter until
// all q.total are taken; units are numbered plan by plan (q.start), the
// caller orders the plans largest first.  The plans share their physics
// (spacing, time step, layer, source), so the time loop takes its
// coefficients from plan 0 (constant-bank operands, as in k_fwd_pair) and
// only the geometry and pointers from the unit's plan.
template <int P, int PR, int NZM, int TOPBC, bool STORE>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1)
k_fwd_pair_queue(const __grid_constant__ QueueArgs q)
{
    __shared__ int unit;
    for (;;) {
        if (threadIdx.x == 0) unit = atomicAdd(q.counter, 1);
        __syncthreads();
        const int u = unit;
        __syncthreads();   // every thread has read it before thread 0 draws again
        if (u >= q.total) return;
        int p = 0;
        while (p + 1 < q.n && u >= q.start[p + 1]) ++p;
        fwd_pair_unit<P, PR, NZM, TOPBC, STORE, false>(q.a[p], q.a[0], u - q.start[p]);
        __syncthreads();   // shared memory is reset by the next unit
    }
}

// ------------------------------------------------------------------ adjoint
// Returns x through an opaque move: values derived from it inside the time
// loop are recomputed every step instead of being hoisted out of the loop
// (22 rows x 2 damping coefficients would pin 44 registers).
__device__ __forceinline__ float opaque(float x)
{
    float y;
    asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int P, int PR, int TOPBC>
__device__ __forceinline__ void adj_rows(const float *__restrict__ cp, float *__restrict__ np,
                                         const float *__restrict__ kp,
                                         const float *__restrict__ sr, float zbf, float ex,
                                         bool top_strip,
                                         bool active, float (&acc)[ROWS], float (&sv)[ROWS],
                                         const PropArgs &a)
{
    float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const float *c = cp + r * P;
        const float wp2 = c[2 * P];
        float lap = a.c0 * w0;
        lap = fmaf(a.cx1, c[-1] + c[1], lap);
        lap = fmaf(a.cx2, c[-2] + c[2], lap);
        lap = fmaf(a.cz1, wm1 + wp1, lap);
        lap = fmaf(a.cz2, wm2 + wp2, lap);
        if (TOPBC == 1 && (r == 1 || r == 2)) {
            // transpose of the mirrored top: reflected weights back onto rows 1, 2
            if (top_strip) lap += (r == 1) ? a.cz1 * wm1 + a.cz2 * w0 : a.cz2 * wm2;
        }
        const float e = ex + ez_of(zbf + (float)r, a);
        const float A2 = __fdividef(2.f, 1.f + e);        // 2A
        const float AB = A2 - 1.f;                        // A B = (1-e)/(1+e)
        const float fo = np[r * P];
        const float fn = fmaf(kp[r * P], lap, fmaf(A2, w0, -AB * fo));
        if (active) np[r * P] = fn;
        acc[r] = fmaf(fn, sv[r], acc[r]);
        sv[r] = sr[r * PR];
        wm2 = wm1;
        wm1 = w0;
        w0 = wp1;
        wp1 = wp2;
    }
}

template <int P, int PR, int NZM, int TOPBC>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1) k_adj_fast(const __grid_constant__ PropArgs a)
{
    extern __shared__ float sm[];
    constexpr int FSZ = (NZM + 4) * P;
    float *U0 = sm, *U1 = sm + FSZ, *K = sm + 2 * FSZ, *IC = K + NZM * P, *ST = IC + a.nr;
    float *RS = ST + a.chunk * a.nr;
    const int NX = a.NX, NZ = a.NZ;
    const int bs = blockIdx.x, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < 2 * FSZ; i += nth) sm[i] = 0.f;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    // kappa / B at each receiver cell (its adjoint source enters through the
    // old level, see below)
    for (int i = tid; i < a.nr; i += nth) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        const float vv = vb[min(rz, a.nz - 1) * a.nx + min(max(rx - a.nb, 0), a.nx - 1)];
        const double vdt = (double)vv * a.dtd;
        IC[i] = (float)(vdt * vdt / (1.0 - e_cell(rx, rz, a)));
    }
    int bad = 0;
    for (int i = tid; i < NZM * P; i += nth) {
        const int pz = i / P, px = i - (i / P) * P;
        float k = 0.f;
        if (pz < NZ && px < NX) {
            const float vv = vb[min(pz, a.nz - 1) * a.nx + min(max(px - a.nb, 0), a.nx - 1)];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, px, pz, a);
        }
        K[i] = k;   // kappa A per cell (0 outside the grid: dead rows stay zero)
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
        return;
    }

    // inactive threads (past the last strip) run the same instructions on the
    // addresses of strip 0, column 0, with every write gated
    const int strip = tid / NX;
    const bool active = strip < a.nstrip;
    const int x = active ? tid % NX : 0;
    const int z0 = active ? strip * ROWS : 0;
    const float ex = ex_of(x, a);
    const float zbf = (float)(z0 - (a.nz - 1));
    const bool top_strip = active && z0 == 0;

    // receiver owned by this thread: its adjoint source enters through the
    // old level, psi^{j-1} -= (kappa / B) q (recomputed where used, to keep
    // the loop-carried state small)
    int inj_slot = -1;
    for (int i = 0; i < a.nr; ++i) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        if (active && x == rx && rz >= z0 && rz < z0 + ROWS) inj_slot = i;
    }
    // source cell: its imaging term sum_j psi^{j+1} s^{nt-1-j} is kept apart
    // (in shared memory, thread 0) because the forward record holds L u only
    __shared__ float acc_src;
    if (tid == 0) acc_src = 0.f;

    const size_t plane = (size_t)a.nzs * PR;   // record planes use the pitch PR
    const int jb = a.j_begin;
    float acc[ROWS], sv[ROWS];
    // record plane read next: starts at forward step nt-1-jb, moves back one
    // plane per step
    const float *sr = a.snap +
                      ((size_t)bs * a.rec_planes + (a.nt - 1 - jb - a.rec_base)) * plane +
                      z0 * PR + x;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        acc[r] = 0.f;
        sv[r] = sr[r * PR];
    }
    if (jb > 0) {
        // resume: levels psi^jb, psi^(jb-1) (a flat copy: per-owner copies
        // of the levels cost registers in the time loop) and the imaging sums
        const size_t cells = (size_t)NZ * NX;
        const float *st = a.astate + (size_t)bs * 3 * cells;
        float *cur = (jb & 1) ? U1 : U0, *old = (jb & 1) ? U0 : U1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            cur[(z + 2) * P + xx + 2] = st[i];
            old[(z + 2) * P + xx + 2] = st[cells + i];
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int z = z0 + r;
                if (z < NZ) acc[r] = st[2 * cells + z * NX + x];
            }
        }
        if (tid == 0) acc_src = a.asrc[bs];
    }
    __syncthreads();

    for (int j0 = jb; j0 < a.j_end; j0 += a.chunk) {
        const int nch = min(a.chunk, a.j_end - j0);
        const float *ab = a.adj + (size_t)bs * a.nr * a.nt;
        for (int e = tid; e < nch * a.nr; e += nth) {
            const int i = e / nch, jj = e - (e / nch) * nch;
            ST[jj * a.nr + i] = IC[i] * ab[(size_t)i * a.nt + (a.nt - 1 - (j0 + jj))];
        }
        // source wavelet of the chunk (source-cell imaging term, thread 0)
        for (int e = tid; e < nch; e += nth) RS[e] = ricker_scaled(a.nt - 1 - (j0 + e), a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (inj_slot >= 0) {
                const int rz = a.rec_pz[inj_slot], rx = a.rec_px[inj_slot];
                nxt[(rz + 2) * P + rx + 2] -= ST[jj * a.nr + inj_slot];   // (kappa/B) q
            }
            if (j + 1 < a.j_end) sr -= plane;
            const float *cp = cur + (z0 + 2) * P + x + 2;
            float *np = nxt + (z0 + 2) * P + x + 2;
            const float *kp = K + z0 * P + x;
            adj_rows<P, PR, TOPBC>(cp, np, kp, sr, opaque(zbf), opaque(ex), top_strip, active, acc, sv,
                               a);
            __syncthreads();
            if (tid == nth - 1) {   // (its warp holds no receivers of the top rows)
                const int sz = a.src_pz[s], sx = a.src_px[s];
                acc_src = fmaf(nxt[(sz + 2) * P + sx + 2], RS[jj], acc_src);
            }
        }
        __syncthreads();   // the last step's source-cell term reads RS before it is restaged
    }

    __syncthreads();
    if (a.j_end < a.nt) {
        // suspend: levels psi^je, psi^(je-1) and the imaging sums
        const int je = a.j_end;
        const size_t cells = (size_t)NZ * NX;
        float *st = a.astate + (size_t)bs * 3 * cells;
        const float *cur = (je & 1) ? U1 : U0, *old = (je & 1) ? U0 : U1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            st[i] = cur[(z + 2) * P + xx + 2];
            st[cells + i] = old[(z + 2) * P + xx + 2];
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int z = z0 + r;
                if (z < NZ) st[2 * cells + z * NX + x] = acc[r];
            }
        }
        if (tid == 0) a.asrc[bs] = acc_src;
        return;
    }

    // dJ/dv_pad = 2 acc / v_pad, fold of the absorbing layer onto the edge
    // cells (transpose of the edge replication), then per-shot gradient
    float *G = U0;   // [NZ][NX]
    float *T = U1;   // [NZ][nx]
    if (active) {
        const int ixc = min(max(x - a.nb, 0), a.nx - 1);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int z = z0 + r;
            if (z < NZ) G[z * NX + x] = 2.f * acc[r] / vb[min(z, a.nz - 1) * a.nx + ixc];
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int sz = a.src_pz[s], sx = a.src_px[s];
        const float vsrc = vb[min(sz, a.nz - 1) * a.nx + min(max(sx - a.nb, 0), a.nx - 1)];
        G[sz * NX + sx] += 2.f * acc_src / vsrc;
    }
    __syncthreads();
    for (int i = tid; i < NZ * a.nx; i += nth) {
        const int pz = i / a.nx, ix = i - (i / a.nx) * a.nx;
        const int c0 = (ix == 0) ? 0 : ix + a.nb;
        const int c1 = (ix == a.nx - 1) ? NX - 1 : ix + a.nb;
        float sum = 0.f;
        for (int px = c0; px <= c1; ++px) sum += G[pz * NX + px];
        T[i] = sum;
    }
    __syncthreads();
    float *gs = a.gshot + (size_t)bs * a.nz * a.nx;
    for (int i = tid; i < a.nz * a.nx; i += nth) {
        const int iz = i / a.nx, ix = i - (i / a.nx) * a.nx;
        const int r1 = (iz == a.nz - 1) ? NZ - 1 : iz;
        float sum = 0.f;
        for (int pz = iz; pz <= r1; ++pz) sum += T[pz * a.nx + ix];
        gs[i] = sum;
    }
}

// ------------------------------------------------------------------ adjoint, column pairs
// k_adj_fast with the column-pair ownership of k_fwd_pair: each thread owns
// columns (x, x+1) x 11 rows, moves them as float2 and updates both columns
// with the packed f32x2 instructions.  Per column the operations and their
// order are those of adj_rows, so the results are bitwise k_adj_fast's
// (the mirrored-top correction apart, whose two products k_adj_fast leaves
// to the compiler's contraction).  A thread may own the receivers of both
// of its columns (one per column and strip).
//
// Registers bound this kernel (unconstrained it wants 140 a thread, and 768
// threads get 80), so the per-cell arrays live in tensor memory instead: the
// imaging sums (read, updated and written back per row) and, side by side,
// kappa A and the damping factor 2A = 2 / (1 + e) (one 4-column read per
// row, which replaces the per-row damping arithmetic: two approximate
// divisions and the layer profile), each thread in its own TMEM lane -- warp
// w owns lanes 32 (w mod 4) .. + 31, the warps of one lane quarter take 68
// columns each (24 of sums, 44 of kappa A and 2A).  The kappa A table in
// shared memory is read only at set-up.
//
// Record reads: a whole record plane is prefetched into L2 two steps before
// it is used (one bulk prefetch per step, in 4 KB pieces), and each thread
// keeps a ring of KR rows in flight (the record of row r + KR is loaded when
// row r is updated).  KR = 6 measured fastest once the sums and kappa A left
// the registers (13.6 ms at 152 models; 4 rows: 14.5 ms).
constexpr int KR = 6;
constexpr int kAdjSumCols = 24;     // a warp's imaging sums: 2 x 11 rows, padded to 4
constexpr int kAdjWarpCols = kAdjSumCols + 4 * ROWS2;   // + (kappa A, 2A) of two cells a row
constexpr int kAdjTmemCols = 512;   // 6 warps per lane quarter x 68 columns, rounded up

// One (model, shot) unit bs of a plan: the whole adjoint time loop of the
// column-pair kernel with its epilogue; `tmem` is the CTA's tensor-memory
// allocation of kAdjTmemCols columns (k_adj_pair allocates it for its one
// unit, k_adj_pair_queue once for all the units it draws)
template <int P, int PR, int NZM, int TOPBC>
__device__ __forceinline__ void adj_pair_unit(const PropArgs &a, const PropArgs &c, const int bs,
                                              const uint32_t tmem)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int FSZ = (NZM + 4) * P;
    static_assert(P % 2 == 0 && PR % 4 == 0 && FSZ % 2 == 0,
                  "float2 rows need even pitches; record planes are prefetched in 16-byte units");
    static_assert(kAdjWarpCols * (kMaxThreadsAdj / 128) <= kAdjTmemCols,
                  "the lane quarters' columns must fit the allocation");
    float *U0 = sm, *U1 = sm + FSZ, *K = sm + 2 * FSZ, *IC = K + NZM * P, *ST = IC + a.nr;
    float *RS = ST + a.chunk * a.nr;
    const int NX = a.NX, NZ = a.NZ;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < 2 * FSZ; i += nth) sm[i] = 0.f;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    // kappa / B at each receiver cell (its adjoint source enters through the
    // old level)
    for (int i = tid; i < a.nr; i += nth) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        const float vv = vb[min(rz, a.nz - 1) * a.nx + min(max(rx - a.nb, 0), a.nx - 1)];
        const double vdt = (double)vv * a.dtd;
        IC[i] = (float)(vdt * vdt / (1.0 - e_cell(rx, rz, a)));
    }
    int bad = 0;
    for (int i = tid; i < NZM * P; i += nth) {
        const int pz = i / P, px = i - (i / P) * P;
        float k = 0.f;
        if (pz < NZ && px < NX) {
            const float vv = vb[min(pz, a.nz - 1) * a.nx + min(max(px - a.nb, 0), a.nx - 1)];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, px, pz, a);
        }
        K[i] = k;   // kappa A per cell (0 outside the grid: dead rows stay zero)
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
        return;
    }

    // inactive threads (past the last strip) run the same instructions on the
    // addresses of strip 0, columns 0 and 1, with every write gated (the
    // tensor-memory accesses are warp-collective)
    const int NXP = NX / 2;
    const int strip = tid / NXP;
    const bool active = strip < a.nstrip;
    const int x = active ? 2 * (tid % NXP) : 0;
    const int z0 = active ? strip * ROWS2 : 0;
    const bool top_strip = active && z0 == 0;

    // receivers owned by this thread (one per column at most)
    int inj0 = -1, inj1 = -1;
    for (int i = 0; i < a.nr; ++i) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        if (active && rz >= z0 && rz < z0 + ROWS2) {
            if (rx == x) inj0 = i;
            if (rx == x + 1) inj1 = i;
        }
    }
    const int inj0_off = inj0 >= 0 ? (a.rec_pz[inj0] + 2) * P + x + 2 : 0;
    const int inj1_off = inj1 >= 0 ? (a.rec_pz[inj1] + 2) * P + x + 3 : 0;
    __shared__ float acc_src;
    if (tid == 0) acc_src = 0.f;
    const int warp = tid >> 5;
    const uint32_t tacc = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                          (uint32_t)(kAdjWarpCols * (warp >> 2));
    const uint32_t tkd = tacc + kAdjSumCols;

    const size_t plane = (size_t)a.nzs * PR;
    const int jb = a.j_begin;
    // record plane of adjoint step j: forward step nt-1-j
    const float *plane_jb =
        a.snap + ((size_t)bs * a.rec_planes + (a.nt - 1 - jb - a.rec_base)) * plane;
    const float *sr = plane_jb + z0 * PR + x;
    // imaging sums (zero, or resumed) and kappa A into this thread's TMEM lane
    // (sizes are recomputed where used: a value live across the time loop
    // costs the loop a register)
#pragma unroll
    for (int r = 0; r < ROWS2; ++r) {
        float2 acc0 = make_float2(0.f, 0.f);
        const int z = z0 + r;
        if (jb > 0 && active && z < NZ) {
            const size_t cells = (size_t)NZ * NX;
            acc0 = f2::ld(a.astate + (size_t)bs * 3 * cells + 2 * cells + z * NX + x);
        }
        tmem_st2(tacc + 2 * r, acc0);
        // 2A = 2 / (1 + e) of the two cells, e = e_x + e_z (side and bottom layer)
        const float ez = ez_of((float)(z0 - (a.nz - 1)) + (float)r, c);
        const float2 h = f2::add(f2::splat(1.f),
                                 f2::add(make_float2(ex_of(x, a), ex_of(x + 1, a)), f2::splat(ez)));
        tmem_st4(tkd + 4 * r, f2::ld(K + z * P + x),
                 make_float2(__fdividef(2.f, h.x), __fdividef(2.f, h.y)));
    }
    tmem_wait_st();
    float2 rq[KR];
#pragma unroll
    for (int i = 0; i < KR; ++i) rq[i] = f2::ld(sr + i * PR);
    if (jb + 1 < a.j_end) prefetch_plane_l2(plane_jb - plane, plane * 4, tid);
    if (jb > 0) {
        // resume: levels psi^jb, psi^(jb-1) and the source-cell sum
        const size_t cells = (size_t)NZ * NX;
        const float *st = a.astate + (size_t)bs * 3 * cells;
        float *cur = (jb & 1) ? U1 : U0, *old = (jb & 1) ? U0 : U1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            cur[(z + 2) * P + xx + 2] = st[i];
            old[(z + 2) * P + xx + 2] = st[cells + i];
        }
        if (tid == 0) acc_src = a.asrc[bs];
    }
    __syncthreads();

    for (int j0 = jb; j0 < a.j_end; j0 += a.chunk) {
        const int nch = min(a.chunk, a.j_end - j0);
        const float *ab = a.adj + (size_t)bs * a.nr * a.nt;
        for (int e = tid; e < nch * a.nr; e += nth) {
            const int i = e / nch, jj = e - (e / nch) * nch;
            ST[jj * a.nr + i] = IC[i] * ab[(size_t)i * a.nt + (a.nt - 1 - (j0 + jj))];
        }
        for (int e = tid; e < nch; e += nth) RS[e] = ricker_scaled(a.nt - 1 - (j0 + e), c);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (inj0 >= 0) nxt[inj0_off] -= ST[jj * a.nr + inj0];   // (kappa/B) q
            if (inj1 >= 0) nxt[inj1_off] -= ST[jj * a.nr + inj1];
            if (j + 2 < a.j_end)
                prefetch_plane_l2(plane_jb - (size_t)(j - jb + 2) * plane, plane * 4, tid);
            const float *sr_next = (j + 1 < a.j_end) ? sr - plane : sr;
            adj_rows_pair<P, PR, ROWS2, KR, TOPBC>(cur + (z0 + 2) * P + x + 2, nxt + (z0 + 2) * P + x + 2,
                                        sr, sr_next, top_strip, active, tacc, tkd, rq, c);
            tmem_wait_st();
            sr = sr_next;
            __syncthreads();
            if (tid == nth - 1) {   // (its warp holds no receivers of the top rows)
                const int sz = a.src_pz[s], sx = a.src_px[s];
                acc_src = fmaf(nxt[(sz + 2) * P + sx + 2], RS[jj], acc_src);
            }
        }
        __syncthreads();   // the last step's source-cell term reads RS before it is restaged
    }

    // the imaging sums back into registers (each thread reads only its own
    // lane and columns, so the next unit may write them at once)
    float2 acc[ROWS2];
#pragma unroll
    for (int r = 0; r < ROWS2; ++r) {
        uint32_t s0, s1;
        tmem_ld2(tacc + 2 * r, s0, s1);
        tmem_wait_ld();
        acc[r] = make_float2(__uint_as_float(s0), __uint_as_float(s1));
    }
    if (a.j_end < a.nt) {
        // suspend: levels psi^je, psi^(je-1) and the imaging sums
        const int je = a.j_end;
        const size_t cells = (size_t)NZ * NX;
        float *st = a.astate + (size_t)bs * 3 * cells;
        const float *cur = (je & 1) ? U1 : U0, *old = (je & 1) ? U0 : U1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            st[i] = cur[(z + 2) * P + xx + 2];
            st[cells + i] = old[(z + 2) * P + xx + 2];
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < ROWS2; ++r) {
                const int z = z0 + r;
                if (z < NZ) f2::st(st + 2 * cells + z * NX + x, acc[r]);
            }
        }
        if (tid == 0) a.asrc[bs] = acc_src;
        return;
    }

    // dJ/dv_pad = 2 acc / v_pad, fold of the absorbing layer onto the edge
    // cells (transpose of the edge replication), then per-shot gradient
    float *G = U0;   // [NZ][NX]
    float *T = U1;   // [NZ][nx]
    if (active) {
        const int ix0 = min(max(x - a.nb, 0), a.nx - 1), ix1 = min(max(x + 1 - a.nb, 0), a.nx - 1);
#pragma unroll
        for (int r = 0; r < ROWS2; ++r) {
            const int z = z0 + r;
            if (z < NZ) {
                const float *vrow = vb + min(z, a.nz - 1) * a.nx;
                G[z * NX + x] = 2.f * acc[r].x / vrow[ix0];
                G[z * NX + x + 1] = 2.f * acc[r].y / vrow[ix1];
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int sz = a.src_pz[s], sx = a.src_px[s];
        const float vsrc = vb[min(sz, a.nz - 1) * a.nx + min(max(sx - a.nb, 0), a.nx - 1)];
        G[sz * NX + sx] += 2.f * acc_src / vsrc;
    }
    __syncthreads();
    for (int i = tid; i < NZ * a.nx; i += nth) {
        const int pz = i / a.nx, ix = i - (i / a.nx) * a.nx;
        const int c0 = (ix == 0) ? 0 : ix + a.nb;
        const int c1 = (ix == a.nx - 1) ? NX - 1 : ix + a.nb;
        float sum = 0.f;
        for (int px = c0; px <= c1; ++px) sum += G[pz * NX + px];
        T[i] = sum;
    }
    __syncthreads();
    float *gs = a.gshot + (size_t)bs * a.nz * a.nx;
    for (int i = tid; i < a.nz * a.nx; i += nth) {
        const int iz = i / a.nx, ix = i - (i / a.nx) * a.nx;
        const int r1 = (iz == a.nz - 1) ? NZ - 1 : iz;
        float sum = 0.f;
        for (int pz = iz; pz <= r1; ++pz) sum += T[pz * a.nx + ix];
        gs[i] = sum;
    }
}

// the CTA's tensor memory for the pair adjoint (one warp allocates; every
// thread sees the base address after the barrier)
template <int P, int PR, int NZM, int TOPBC>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1) k_adj_pair(const __grid_constant__ PropArgs a)
{
    __shared__ uint32_t tmem_slot;
    const uint32_t tmem = tmem_alloc(&tmem_slot, kAdjTmemCols);
    adj_pair_unit<P, PR, NZM, TOPBC>(a, a, blockIdx.x, tmem);
    tmem_free(tmem, kAdjTmemCols);
}

// Persistent: units drawn from the counter as in k_fwd_pair_queue, one
// tensor-memory allocation for all of them
template <int P, int PR, int NZM, int TOPBC>
__global__ void __launch_bounds__(kMaxThreadsAdj, 1)
k_adj_pair_queue(const __grid_constant__ QueueArgs q)
{
    __shared__ uint32_t tmem_slot;
    __shared__ int unit;
    const uint32_t tmem = tmem_alloc(&tmem_slot, kAdjTmemCols);
    for (;;) {
        if (threadIdx.x == 0) unit = atomicAdd(q.counter, 1);
        __syncthreads();
        const int u = unit;
        __syncthreads();
        if (u >= q.total) break;
        int p = 0;
        while (p + 1 < q.n && u >= q.start[p + 1]) ++p;
        adj_pair_unit<P, PR, NZM, TOPBC>(q.a[p], q.a[0], u - q.start[p], tmem);
        __syncthreads();
    }
    tmem_free(tmem, kAdjTmemCols);
}

template <typename K>
cudaError_t launch_k(K kern, const PropArgs &a, const ResidentShape &sh, int nblocks,
                     cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh.smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, sh.threads, sh.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Buckets of the fast kernels: shared-memory pitch P, record pitch PR and
// row capacity NZM.  P = 1 (mod 16) shifts the banks of the next 22-row strip
// by 22 words, which keeps the warps that straddle two strips free of bank
// conflicts at 150 padded columns (5 strips of 150 threads); the record
// planes keep a multiple-of-32 pitch so that their rows stay 128-byte aligned.
bool fast_bucket(int NZ, int NX, int *P, int *PR, int *NZM)
{
    static const int buckets[][3] = {{65, 64, 264}, {161, 160, 110}};
    for (const auto &bk : buckets) {
        const int p = bk[0], pr = bk[1], nzm = bk[2];
        if (NX + 4 > pr || NZ > nzm) continue;
        const int nstrip = (NZ + kFastRows - 1) / kFastRows;
        if (NX * nstrip > kMaxThreadsAdj) continue;
        *P = p;
        *PR = pr;
        *NZM = nzm;
        return true;
    }
    return false;
}

bool fwd_pair_ok(int NX, int NZ, int NZM)
{
    const int nstrip = (NZ + kFastRows / 2 - 1) / (kFastRows / 2);
    return NZM == 110 && NX % 2 == 0 && NX + 4 <= 160 && (NX / 2) * nstrip <= kMaxThreadsAdj;
}

size_t fast_smem(int P, int NZM, bool adj, int chunk, int nr)
{
    // two field levels + one per-cell table (A B for the forward, kappa A for
    // the adjoint) + the adjoint's per-receiver coefficients + the staging
    // chunk (receiver samples; the adjoint also stages the source wavelet)
    return ((size_t)2 * (NZM + 4) * P + (size_t)NZM * P + (adj ? (size_t)nr : 0) +
            (size_t)chunk * (nr + (adj ? 1 : 0))) * sizeof(float);
}

int fast_chunk(int P, int NZM, bool adj, int nr)
{
    const size_t limit = 227 * 1024, fixed = fast_smem(P, NZM, adj, 0, nr);
    const size_t per = ((size_t)nr + (adj ? 1 : 0)) * sizeof(float);
    if (fixed + per > limit) return 0;
    const size_t c = (limit - fixed) / per;
    return c > 32 ? 32 : (int)c;
}

bool queue_same_physics(const Plan &a, const Plan &b)
{
    const fwi_problem &p = a.p, &q = b.p;
    return p.dx == q.dx && p.dz == q.dz && p.dt == q.dt && p.nb == q.nb && p.top_bc == q.top_bc &&
           p.v_ref == q.v_ref && p.refl_R == q.refl_R && p.f_peak == q.f_peak && a.t0 == b.t0;
}

bool queue_ok(const Plan &pl)
{
    return pl.fast && pl.fwd_pair && pl.adj_pair && pl.fast_NZM == 110 && pl.ckpt_every == 0 &&
           !pl.cpml;
}

cudaError_t launch_fast_queue(const Plan *const *plans, int n, bool adj, const PropArgs *a,
                              int *counter, cudaStream_t st)
{
    if (n < 1 || n > kQueuePlans) return cudaErrorInvalidValue;
    QueueArgs q{};
    q.n = n;
    q.counter = counter;
    size_t smem = 0;
    const int tb = plans[0]->p.top_bc;
    for (int i = 0; i < n; ++i) {
        const Plan &pl = *plans[i];
        if (!queue_ok(pl) || !queue_same_physics(pl, *plans[0])) return cudaErrorInvalidValue;
        const ResidentShape &sh = adj ? pl.shape_adj : pl.shape;
        q.start[i] = q.total;
        q.total += pl.p.batch * pl.p.ns;
        q.a[i] = a[i];
        q.a[i].rows = sh.rows;
        q.a[i].nstrip = sh.nstrip;
        q.a[i].chunk = sh.chunk;
        if (sh.smem > smem) smem = sh.smem;
    }
    q.start[n] = q.total;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int grid = q.total < sms ? q.total : sms;
    auto go = [&](auto kern) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r != cudaSuccess) return r;
        kern<<<grid, kMaxThreadsAdj, smem, st>>>(q);
        return cudaGetLastError();
    };
    const bool store = a[0].snap != nullptr;
    if (adj) return tb ? go(k_adj_pair_queue<kPairPitch, 160, 110, 1>)
                       : go(k_adj_pair_queue<kPairPitch, 160, 110, 0>);
    if (store) return tb ? go(k_fwd_pair_queue<kPairPitch, 160, 110, 1, true>)
                         : go(k_fwd_pair_queue<kPairPitch, 160, 110, 0, true>);
    return tb ? go(k_fwd_pair_queue<kPairPitch, 160, 110, 1, false>)
              : go(k_fwd_pair_queue<kPairPitch, 160, 110, 0, false>);
}

cudaError_t launch_fast(const Plan &pl, bool adj, const PropArgs &a, cudaStream_t st)
{
    const int nb = pl.p.batch * pl.p.ns;
    const ResidentShape &sh = adj ? pl.shape_adj : pl.shape;
    const bool store = a.snap != nullptr;
    const int tb = pl.p.top_bc;
#define FWI_FAST(PP, PPR, NN)                                                                  \
    if (pl.fast_P == PP && pl.fast_NZM == NN) {                                                \
        if (adj)                                                                               \
            return tb ? launch_k(k_adj_fast<PP, PPR, NN, 1>, a, sh, nb, st)                    \
                      : launch_k(k_adj_fast<PP, PPR, NN, 0>, a, sh, nb, st);                   \
        if (store)                                                                             \
            return tb ? launch_k(k_fwd_fast<PP, PPR, NN, 1, true>, a, sh, nb, st)              \
                      : launch_k(k_fwd_fast<PP, PPR, NN, 0, true>, a, sh, nb, st);             \
        return tb ? launch_k(k_fwd_fast<PP, PPR, NN, 1, false>, a, sh, nb, st)                 \
                  : launch_k(k_fwd_fast<PP, PPR, NN, 0, false>, a, sh, nb, st);                \
    }
    if (adj && pl.adj_pair) {
        if (pl.fast_NZM == 110)
            return tb ? launch_k(k_adj_pair<kPairPitch, 160, 110, 1>, a, sh, nb, st)
                      : launch_k(k_adj_pair<kPairPitch, 160, 110, 0>, a, sh, nb, st);
        return cudaErrorInvalidValue;
    }
    if (!adj && pl.fwd_pair) {
        if (pl.fast_NZM == 110)
            return store ? (tb ? launch_k(k_fwd_pair<kPairPitch, 160, 110, 1, true>, a, sh, nb, st)
                               : launch_k(k_fwd_pair<kPairPitch, 160, 110, 0, true>, a, sh, nb, st))
                         : (tb ? launch_k(k_fwd_pair<kPairPitch, 160, 110, 1, false>, a, sh, nb, st)
                               : launch_k(k_fwd_pair<kPairPitch, 160, 110, 0, false>, a, sh, nb, st));
        return cudaErrorInvalidValue;
    }
    FWI_FAST(65, 64, 264)
    FWI_FAST(161, 160, 110)
#undef FWI_FAST
    return cudaErrorInvalidValue;
}

}  // namespace fwi
