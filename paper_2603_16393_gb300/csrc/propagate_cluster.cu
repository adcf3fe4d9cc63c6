// propagate_cluster.cu -- propagators for padded grids too large for one
// CTA's shared memory but small enough for a cluster's (for example 256 x 256
// models with a 40-cell layer: 296 x 336 cells).
//
// The grid of a (model, shot) is split by rows across a cluster of C CTAs
// (2 <= C <= 8, a launch attribute): CTA c keeps rows [c RC, (c+1) RC) of
// both time levels in its shared memory, with two halo rows above and below.
// RC is a whole number of RS-row thread strips.  After a step, the threads
// of a CTA's first (last) strip put their two edge rows of the new level into
// the bottom (top) halo rows of the CTA above (below) with st.async; each
// store counts its bytes on the receiving CTA's mbarrier for that level, and a
// CTA reads a level's halo rows only once its mbarrier has seen all of them.
// No cluster-wide barrier runs per step, and the fields never leave the chip:
// only the wavefield record, traces and gradients go to HBM.
//
// Ordering, with every CTA's step j ending in its wait for level j+1:
// * a CTA writes level j+1 into a neighbour's buffer that held level j-1,
//   whose halo rows that neighbour read only for its own edge rows of level
//   j; it sent those edge rows (after computing them) before this CTA could
//   finish waiting for level j, which precedes its step j;
// * level L counts on mbarrier L mod 4, armed (expected bytes, one arrival)
//   exactly once: levels 1, 2 before the first step, level L >= 3 at the
//   start of step L-3, which follows the wait for level L-4 on the same
//   mbarrier (end of step L-5) and precedes, by a CTA barrier, this CTA's
//   step L-2 sends of level L-1, without which no neighbour computes level
//   L.  So a phase is armed before any of its bytes arrive, and its bytes
//   arrive after the previous phase ended.
//
// Same recurrences and coefficient formation as the single-CTA resident
// kernels: forward in increment form with a difference Laplacian and the
// FP64-formed A B table; adjoint in the self-adjoint phi = kappa A mu form
// (the receivers' adjoint source through the old level, imaging acc +=
// psi^{j+1} t^{nt-1-j}, source-cell term kept apart), its imaging sums in
// shared memory; they go to the tiled kernels' buffers, whose fold kernel
// finishes.  The record of a cluster plan has C RC rows per plane at the row
// pitch P - 1, so that every record access is a compile-time offset.
//
// Every halo wait is bounded in time; one that runs out sets
// FWI_ERR_DEVICE_TIMEOUT and the CTA stops waiting but runs every remaining
// step, so every CTA reaches the final cluster barrier.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "f32x2.cuh"
#include "fwi_device.cuh"
#include "fwi_internal.cuh"
#include "stencil_pair.cuh"
#include "tmem.cuh"

namespace cg = cooperative_groups;

namespace fwi {

namespace {

constexpr unsigned long long kHaloWaitNs = 2000000000ull;   // 2 s per level
constexpr int kHaloBars = 4;   // level L of the fields counts on mbarrier L mod 4

using dev::e_cell;
using dev::ex_of;
using dev::ez_of;
using dev::kappaA_cell;
using dev::ricker_scaled;

__device__ __forceinline__ unsigned s_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// The same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned at_rank(unsigned addr, int rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// One float into another CTA's shared memory, its 4 bytes counted on that
// CTA's mbarrier.
__device__ __forceinline__ void put_remote(unsigned raddr, float v, unsigned rmbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                     raddr),
                 "r"(__float_as_uint(v)), "r"(rmbar)
                 : "memory");
}

// The single arrival of a phase, with the bytes the neighbours will send.
__device__ __forceinline__ void halo_arm(uint64_t *mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(mb)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool halo_try(uint64_t *mb, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(s_u32(mb)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits (bounded by limit_ns) until the neighbours' halo rows of a level
// have landed.
__device__ __forceinline__ void halo_wait(uint64_t *mb, unsigned parity, volatile int *failed,
                                          int *status, unsigned long long limit_ns)
{
    if (*failed || halo_try(mb, parity)) return;
    const unsigned long long t0 = now_ns();
    while (!halo_try(mb, parity)) {
        if (*failed) return;
        if (now_ns() - t0 > limit_ns) {
            *failed = 1;
            set_status(status, FWI_ERR_DEVICE_TIMEOUT);
            return;
        }
    }
}

// One thread: set up the mbarriers and arm levels 1 and 2 (step j arms level
// j+3, so that every level is armed exactly once).
__device__ __forceinline__ void halo_init(uint64_t *mb, unsigned bytes, int nt)
{
    for (int k = 0; k < kHaloBars; ++k)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(mb + k)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int L = 1; L <= 2 && L <= nt; ++L) halo_arm(mb + L, bytes);
}

// Parity of the mbarrier phase that counts level L >= 1.
__device__ __forceinline__ unsigned halo_parity(int L) { return (unsigned)((L - 1) >> 2) & 1u; }

// Edge rows of the new level (np: this thread's first row) to the neighbours'
// halo rows: rows 0, 1 of a first strip to rows RC, RC+1 of the CTA above,
// rows RS-2, RS-1 of a last strip to rows -2, -1 of the CTA below.
template <int P, int RS>
__device__ __forceinline__ void send_edges(const float *np, int RC, int crank, bool up, bool dn,
                                           uint64_t *mb)
{
    if (up) {
        const unsigned rm = at_rank(s_u32(mb), crank - 1);
        const unsigned ra = at_rank(s_u32(np + RC * P), crank - 1);
        put_remote(ra, np[0], rm);
        put_remote(ra + 4 * P, np[P], rm);
    }
    if (dn) {
        const unsigned rm = at_rank(s_u32(mb), crank + 1);
        const unsigned ra = at_rank(s_u32(np + (RS - 2 - RC) * P), crank + 1);
        put_remote(ra, np[(RS - 2) * P], rm);
        put_remote(ra + 4 * P, np[(RS - 1) * P], rm);
    }
}

template <int P, int RS, int TOPBC, bool STORE>
__global__ void __launch_bounds__(clu_max_threads(RS), 1)
k_clu_fwd(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = e.C, crank = (int)cl.block_rank();
    const int bs = blockIdx.x / C, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (RC + 4) * P;
    extern __shared__ float sm[];
    __shared__ uint64_t mb[kHaloBars];
    __shared__ int failed;
    float *U0 = sm, *U1 = U0 + FS, *ABt = U1 + FS, *ST = ABt + RC * P;
    float *RSw = ST + e.chunk * a.nr;
    const int g0 = crank * RC;                 // first grid row of this CTA
    for (int i = tid; i < 2 * FS; i += nth) sm[i] = 0.f;
    for (int i = tid; i < RC * P; i += nth) {
        const int lr = i / P, px = i - (i / P) * P, gz = g0 + lr;
        float m = 0.f;
        if (gz < NZ && px < NX) {
            const double ee = e_cell(px, gz, a);
            m = (float)((1.0 - ee) / (1.0 + ee));
        }
        ABt[i] = m;
    }
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    const int x = tid % NX, strip = tid / NX;
    const bool active = strip < e.nstrip;
    const int l0 = strip * RS;
    const int ixc = min(max(x - a.nb, 0), a.nx - 1);
    float ka[RS], vi[RS];
    int bad = 0;
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const int gz = g0 + l0 + r;
        float k = 0.f;
        if (active && gz < NZ) {
            const float vv = vb[min(gz, a.nz - 1) * a.nx + ixc];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, x, gz, a);
        }
        ka[r] = k;
        vi[r] = 0.f;
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    const bool has_up = crank > 0, has_dn = crank + 1 < C;
    const bool send_up = active && strip == 0 && has_up;
    const bool send_dn = active && strip == e.nstrip - 1 && has_dn;
    const bool top_strip = active && strip == 0 && crank == 0;
    const unsigned halo_bytes = (unsigned)((has_up ? 1 : 0) + (has_dn ? 1 : 0)) * 8u * NX;
    if (tid == 0) {
        halo_init(mb, halo_bytes, a.nt);
        failed = 0;
    }
    // source owner
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const int src_row = (active && x == sx && sz >= g0 + l0 && sz < g0 + l0 + RS) ? sz - g0 - l0 : -1;
    float ka_src = 0.f;
#pragma unroll
    for (int r = 0; r < RS; ++r)
        if (r == src_row) ka_src = ka[r];
    // record plane of step j: rows [0, C RC) at the compile-time pitch PRC
    constexpr int PRC = P - 1;
    const size_t plane = (size_t)C * RC * PRC;
    float *sw = STORE ? a.snap + (size_t)bs * a.rec_planes * plane + (size_t)(g0 + l0) * PRC + x
                      : nullptr;
    cl.sync();   // every CTA's fields are zero and its mbarriers set up

    for (int j0 = 0; j0 < a.nt; j0 += e.chunk) {
        const int nch = min(e.chunk, a.nt - j0);
        for (int q = tid; q < nch; q += nth) RSw[q] = ricker_scaled(j0 + q, a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            // after a halo wait has run out (the flag only goes 0 -> 1) no phase
            // is armed again: an arm by thread 0 implies its own wait for the
            // barrier's previous phase (level j-1, two steps ago) succeeded
            if (tid == 0 && j + 3 <= a.nt && !*(volatile int *)&failed)
                halo_arm(&mb[(j + 3) & 3], halo_bytes);
            if (active) {
                const float *cp = cur + (l0 + 2) * P + x + 2;
                float *np = nxt + (l0 + 2) * P + x + 2;
                const float *abp = ABt + l0 * P + x;
                float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
                float Dp = w0 - wm1, Em2 = w0 - wm2, Em1 = wp1 - wm1;
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    const float *c = cp + r * P;
                    const float wp2 = c[2 * P];
                    const float Dn = wp1 - w0;
                    const float E0 = wp2 - w0;
                    const float dzA = Dn - Dp;
                    const float dzB = E0 - Em2;
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
                        if (top_strip) np[-r * P] = un;   // mirrored ghost rows -1, -2
                    }
                    if (STORE) sw[r * PRC] = lap;
                    Dp = Dn;
                    Em2 = Em1;
                    Em1 = E0;
                    wm2 = wm1;
                    wm1 = w0;
                    w0 = wp1;
                    wp1 = wp2;
                }
                if (src_row >= 0) {
                    // point source: + kappa A s at the source cell (increment and field)
                    const float d = ka_src * RSw[jj];
#pragma unroll
                    for (int r = 0; r < RS; ++r)
                        if (r == src_row) vi[r] += d;
                    np[src_row * P] += d;
                    if (TOPBC == 1 && top_strip && (src_row == 1 || src_row == 2))
                        np[-src_row * P] += d;
                }
                // a CTA whose wait ran out sends no more halo rows, so that its
                // neighbours' waits run out too, within a level or two
                if (!e.withhold && !*(volatile int *)&failed)
                    send_edges<P, RS>(np, RC, crank, send_up, send_dn, &mb[(j + 1) & 3]);
            }
            if (STORE) sw += plane;
            __syncthreads();
            for (int i = tid; i < a.nr; i += nth) {
                const int rz = a.rec_pz[i] - g0;
                if (rz >= 0 && rz < RC) ST[jj * a.nr + i] = nxt[(rz + 2) * P + a.rec_px[i] + 2];
            }
            // the neighbours' edge rows of level j+1 in this CTA's halo rows
            halo_wait(&mb[(j + 1) & 3], halo_parity(j + 1), &failed, a.status, e.wait_ns);
        }
        __syncthreads();
        float *db = a.d_syn + (size_t)bs * a.nr * a.nt;
        for (int q = tid; q < nch * a.nr; q += nth) {
            const int i = q / nch, jj = q - (q / nch) * nch;
            const int rz = a.rec_pz[i] - g0;
            if (rz >= 0 && rz < RC) db[(size_t)i * a.nt + j0 + jj] = ST[jj * a.nr + i];
        }
        __syncthreads();
    }
    cl.sync();   // no CTA leaves while a neighbour may still write into it
}

template <int P, int RS, int TOPBC>
__global__ void __launch_bounds__(clu_max_threads(RS), 1)
k_clu_adj(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = e.C, crank = (int)cl.block_rank();
    const int bs = blockIdx.x / C, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (RC + 4) * P;
    constexpr int PRC = P - 1;
    extern __shared__ float sm[];
    __shared__ uint64_t mb[kHaloBars];
    __shared__ int failed;
    __shared__ float acc_src;
    // imaging sums acc of this CTA's cells live in shared memory (row pitch PRC)
    float *U0 = sm, *U1 = U0 + FS, *K = U1 + FS, *ACC = K + RC * P, *IC = ACC + RC * PRC;
    float *ST = IC + a.nr, *RSw = ST + e.chunk * a.nr;
    const int g0 = crank * RC;
    for (int i = tid; i < 2 * FS; i += nth) sm[i] = 0.f;
    for (int i = tid; i < RC * PRC; i += nth) ACC[i] = 0.f;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    for (int i = tid; i < a.nr; i += nth) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        const float vv = vb[min(rz, a.nz - 1) * a.nx + min(max(rx - a.nb, 0), a.nx - 1)];
        const double vdt = (double)vv * a.dtd;
        IC[i] = (float)(vdt * vdt / (1.0 - e_cell(rx, rz, a)));   // kappa / B
    }
    int bad = 0;
    for (int i = tid; i < RC * P; i += nth) {
        const int lr = i / P, px = i - (i / P) * P, gz = g0 + lr;
        float k = 0.f;
        if (gz < NZ && px < NX) {
            const float vv = vb[min(gz, a.nz - 1) * a.nx + min(max(px - a.nb, 0), a.nx - 1)];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, px, gz, a);
        }
        K[i] = k;
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    const int x = tid % NX, strip = tid / NX;
    const bool active = strip < e.nstrip;
    const int l0 = strip * RS;
    const float ex = ex_of(x, a);
    const float zbf = (float)(g0 + l0 - (a.nz - 1));
    const bool has_up = crank > 0, has_dn = crank + 1 < C;
    const bool send_up = active && strip == 0 && has_up;
    const bool send_dn = active && strip == e.nstrip - 1 && has_dn;
    const bool top_strip = active && strip == 0 && crank == 0;
    const unsigned halo_bytes = (unsigned)((has_up ? 1 : 0) + (has_dn ? 1 : 0)) * 8u * NX;
    if (tid == 0) {
        halo_init(mb, halo_bytes, a.nt);
        failed = 0;
        acc_src = 0.f;
    }
    // receiver owned by this thread (at most one per column of a strip)
    int inj_slot = -1;
    for (int i = 0; i < a.nr; ++i) {
        const int rz = a.rec_pz[i] - g0, rx = a.rec_px[i];
        if (active && x == rx && rz >= l0 && rz < l0 + RS) inj_slot = i;
    }
    const int inj_off = inj_slot >= 0 ? (a.rec_pz[inj_slot] - g0 + 2) * P + x + 2 : 0;
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const bool src_here = sz >= g0 && sz < g0 + RC;
    const size_t plane = (size_t)C * RC * PRC;
    float sv[RS];
    // record plane read next: forward step nt-1, then one plane back per step
    const float *sr =
        a.snap + ((size_t)bs * a.rec_planes + (a.nt - 1)) * plane + (size_t)(g0 + l0) * PRC + x;
#pragma unroll
    for (int r = 0; r < RS; ++r) sv[r] = active ? sr[r * PRC] : 0.f;
    float *ac = ACC + l0 * PRC + x;
    const float *kp = K + l0 * P + x;
    cl.sync();   // every CTA's fields are zero and its mbarriers set up

    for (int j0 = 0; j0 < a.nt; j0 += e.chunk) {
        const int nch = min(e.chunk, a.nt - j0);
        const float *ab = a.adj + (size_t)bs * a.nr * a.nt;
        for (int q = tid; q < nch * a.nr; q += nth) {
            const int i = q / nch, jj = q - (q / nch) * nch;
            ST[jj * a.nr + i] = IC[i] * ab[(size_t)i * a.nt + (a.nt - 1 - (j0 + jj))];
        }
        for (int q = tid; q < nch; q += nth) RSw[q] = ricker_scaled(a.nt - 1 - (j0 + q), a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            // after a halo wait has run out (the flag only goes 0 -> 1) no phase
            // is armed again: an arm by thread 0 implies its own wait for the
            // barrier's previous phase (level j-1, two steps ago) succeeded
            if (tid == 0 && j + 3 <= a.nt && !*(volatile int *)&failed)
                halo_arm(&mb[(j + 3) & 3], halo_bytes);
            if (inj_slot >= 0) nxt[inj_off] -= ST[jj * a.nr + inj_slot];   // (kappa/B) q
            if (j + 1 < a.nt) sr -= plane;
            if (active) {
                const float *cp = cur + (l0 + 2) * P + x + 2;
                float *np = nxt + (l0 + 2) * P + x + 2;
                float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    const float *c = cp + r * P;
                    const float wp2 = c[2 * P];
                    float lap = a.c0 * w0;
                    lap = fmaf(a.cx1, c[-1] + c[1], lap);
                    lap = fmaf(a.cx2, c[-2] + c[2], lap);
                    lap = fmaf(a.cz1, wm1 + wp1, lap);
                    lap = fmaf(a.cz2, wm2 + wp2, lap);
                    if (TOPBC == 1 && (r == 1 || r == 2)) {
                        // transpose of the mirrored top: reflected weights onto rows 1, 2
                        if (top_strip) lap += (r == 1) ? a.cz1 * wm1 + a.cz2 * w0 : a.cz2 * wm2;
                    }
                    const float ee = ex + ez_of(zbf + (float)r, a);
                    const float A2 = __fdividef(2.f, 1.f + ee);   // 2A
                    const float AB = A2 - 1.f;                     // A B
                    const float fo = np[r * P];
                    const float fn = fmaf(kp[r * P], lap, fmaf(A2, w0, -AB * fo));
                    np[r * P] = fn;
                    ac[r * PRC] = fmaf(fn, sv[r], ac[r * PRC]);
                    sv[r] = sr[r * PRC];
                    wm2 = wm1;
                    wm1 = w0;
                    w0 = wp1;
                    wp1 = wp2;
                }
                // a CTA whose wait ran out sends no more halo rows, so that its
                // neighbours' waits run out too, within a level or two
                if (!e.withhold && !*(volatile int *)&failed)
                    send_edges<P, RS>(np, RC, crank, send_up, send_dn, &mb[(j + 1) & 3]);
            }
            __syncthreads();
            if (tid == nth - 1 && src_here)
                acc_src = fmaf(nxt[(sz - g0 + 2) * P + sx + 2], RSw[jj], acc_src);
            halo_wait(&mb[(j + 1) & 3], halo_parity(j + 1), &failed, a.status, e.wait_ns);
        }
        __syncthreads();
    }
    // imaging sums of this CTA's rows and the source-cell sum to the fold
    for (int i = tid; i < RC * NX; i += nth) {
        const int lr = i / NX, px = i - (i / NX) * NX, gz = g0 + lr;
        if (gz < NZ) e.acc[((size_t)bs * NZ + gz) * e.NXp + px] = ACC[lr * PRC + px];
    }
    if (tid == 0 && src_here) e.acc_src[bs] = acc_src;
    cl.sync();   // no CTA leaves while a neighbour may still write into it
}

// ------------------------------------------------------------------ column pairs
// The same cluster scheme with the column-pair threads of the resident
// kernels: a thread owns columns (x, x+1) x RW rows of its CTA's rows, moves
// them as 8-byte accesses and updates both with packed f32x2 operations
// (stencil_pair.cuh; per cell the operations and their order are those of
// k_clu_fwd / k_clu_adj, so the results are bitwise theirs with the reflecting
// top).  Halo rows go out as 8-byte st.async stores (the same bytes per level
// on each mbarrier).  The adjoint keeps its imaging sums and (kappa A, 2A)
// in tensor memory instead of shared memory and registers, reads the record
// through a ring of KR rows per thread and prefetches its CTA's part of each
// record plane into L2 two steps ahead.
constexpr int kCluKR = 6;
constexpr int kCluSumCols = 24;                               // 2 x 10 sums, padded to 4
constexpr int kCluWarpCols = kCluSumCols + 4 * kCluPairRows;  // + (kappa A, 2A) a row
constexpr int kCluTmemCols = 512;
constexpr size_t kCluSoloSmem = 116 * 1024;   // > half of an SM's 228 KB
static_assert(kCluWarpCols * ((kCluPairThreads / 32 + 3) / 4) <= kCluTmemCols,
              "the lane quarters' columns must fit the allocation");

// two floats into another CTA's shared memory, 8 bytes counted on its mbarrier
__device__ __forceinline__ void put_remote2(unsigned raddr, float2 v, unsigned rmbar)
{
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(
            raddr),
        "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(rmbar)
        : "memory");
}

// send_edges for a column pair (np: the thread's first row, 8-byte aligned)
template <int P, int RW>
__device__ __forceinline__ void send_edges_pair(const float *np, int RC, int crank, bool up,
                                                bool dn, uint64_t *mb)
{
    if (up) {
        const unsigned rm = at_rank(s_u32(mb), crank - 1);
        const unsigned ra = at_rank(s_u32(np + RC * P), crank - 1);
        put_remote2(ra, f2::ld(np), rm);
        put_remote2(ra + 4 * P, f2::ld(np + P), rm);
    }
    if (dn) {
        const unsigned rm = at_rank(s_u32(mb), crank + 1);
        const unsigned ra = at_rank(s_u32(np + (RW - 2 - RC) * P), crank + 1);
        put_remote2(ra, f2::ld(np + (RW - 2) * P), rm);
        put_remote2(ra + 4 * P, f2::ld(np + (RW - 1) * P), rm);
    }
}

template <int P, int RW, int TOPBC, bool STORE>
__global__ void __launch_bounds__(kCluPairThreads, 1)
k_clu_fwd_pair(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = e.C, crank = (int)cl.block_rank();
    const int bs = blockIdx.x / C, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (RC + 4) * P;
    constexpr int PRC = kCluPitch - 1;
    extern __shared__ __align__(16) float sm[];
    __shared__ uint64_t mb[kHaloBars];
    __shared__ int failed;
    float *U0 = sm, *U1 = U0 + FS, *ABt = U1 + FS, *ST = ABt + RC * P;
    float *RSw = ST + e.chunk * a.nr;
    const int g0 = crank * RC;
    for (int i = tid; i < 2 * FS; i += nth) sm[i] = 0.f;
    for (int i = tid; i < RC * P; i += nth) {
        const int lr = i / P, px = i - (i / P) * P, gz = g0 + lr;
        float m = 0.f;
        if (gz < NZ && px < NX) {
            const double ee = e_cell(px, gz, a);
            m = (float)((1.0 - ee) / (1.0 + ee));
        }
        ABt[i] = m;
    }
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    const int NXP = NX / 2;
    const int xp = tid % NXP, strip = tid / NXP;
    const bool active = strip < e.nstrip;
    const int x = 2 * xp, l0 = strip * RW;
    float2 ka[RW], vi[RW];
    int bad = 0;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int gz = g0 + l0 + r;
        float k[2] = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (active && gz < NZ) {
                const float vv = vb[min(gz, a.nz - 1) * a.nx + min(max(x + c - a.nb, 0), a.nx - 1)];
                if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
                k[c] = kappaA_cell(vv, x + c, gz, a);
            }
        }
        ka[r] = make_float2(k[0], k[1]);
        vi[r] = make_float2(0.f, 0.f);
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    const bool has_up = crank > 0, has_dn = crank + 1 < C;
    const bool send_up = active && strip == 0 && has_up;
    const bool send_dn = active && strip == e.nstrip - 1 && has_dn;
    const bool top_strip = active && strip == 0 && crank == 0;
    const unsigned halo_bytes = (unsigned)((has_up ? 1 : 0) + (has_dn ? 1 : 0)) * 8u * NX;
    if (tid == 0) {
        halo_init(mb, halo_bytes, a.nt);
        failed = 0;
    }
    // source owner: row and column inside this thread's RW x 2 block
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const int src_k = (active && (sx >> 1) == xp && sz >= g0 + l0 && sz < g0 + l0 + RW)
                          ? 2 * (sz - g0 - l0) + (sx & 1) : -1;
    float kas = 0.f;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        if (2 * k == src_k) kas = ka[k].x;
        if (2 * k + 1 == src_k) kas = ka[k].y;
    }
    const size_t plane = (size_t)C * RC * PRC;
    float *sw = STORE ? a.snap + (size_t)bs * a.rec_planes * plane + (size_t)(g0 + l0) * PRC + x
                      : nullptr;
    cl.sync();   // every CTA's fields are zero and its mbarriers set up

    for (int j0 = 0; j0 < a.nt; j0 += e.chunk) {
        const int nch = min(e.chunk, a.nt - j0);
        for (int q = tid; q < nch; q += nth) RSw[q] = ricker_scaled(j0 + q, a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            // after a halo wait has run out (the flag only goes 0 -> 1) no phase
            // is armed again (see k_clu_fwd)
            if (tid == 0 && j + 3 <= a.nt && !*(volatile int *)&failed)
                halo_arm(&mb[(j + 3) & 3], halo_bytes);
            if (active) {
                const float *cp = cur + (l0 + 2) * P + x + 2;
                float *np = nxt + (l0 + 2) * P + x + 2;
                fwd_rows_pair<P, PRC, RW, TOPBC, STORE, true>(cp, np, ABt + l0 * P + x, sw,
                                                               top_strip, ka, vi, a);
                if (src_k >= 0) {
                    // point source: + kappa A s at the source cell (increment and field)
                    const float d = kas * RSw[jj];
#pragma unroll
                    for (int k = 0; k < RW; ++k) {
                        if (2 * k == src_k) vi[k].x += d;
                        if (2 * k + 1 == src_k) vi[k].y += d;
                    }
                    const int lz = sz - g0;
                    nxt[(lz + 2) * P + sx + 2] += d;
                    if (TOPBC == 1 && crank == 0 && (lz == 1 || lz == 2))
                        nxt[(2 - lz) * P + sx + 2] += d;
                }
                // a CTA whose wait ran out sends no more halo rows
                if (!e.withhold && !*(volatile int *)&failed)
                    send_edges_pair<P, RW>(np, RC, crank, send_up, send_dn, &mb[(j + 1) & 3]);
            }
            if (STORE) sw += plane;
            __syncthreads();
            for (int i = tid; i < a.nr; i += nth) {
                const int rz = a.rec_pz[i] - g0;
                if (rz >= 0 && rz < RC) ST[jj * a.nr + i] = nxt[(rz + 2) * P + a.rec_px[i] + 2];
            }
            halo_wait(&mb[(j + 1) & 3], halo_parity(j + 1), &failed, a.status, e.wait_ns);
        }
        __syncthreads();
        float *db = a.d_syn + (size_t)bs * a.nr * a.nt;
        for (int q = tid; q < nch * a.nr; q += nth) {
            const int i = q / nch, jj = q - (q / nch) * nch;
            const int rz = a.rec_pz[i] - g0;
            if (rz >= 0 && rz < RC) db[(size_t)i * a.nt + j0 + jj] = ST[jj * a.nr + i];
        }
        __syncthreads();
    }
    cl.sync();   // no CTA leaves while a neighbour may still write into it
}

template <int P, int RW, int TOPBC>
__global__ void __launch_bounds__(kCluPairThreads, 1)
k_clu_adj_pair(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = e.C, crank = (int)cl.block_rank();
    const int bs = blockIdx.x / C, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (RC + 4) * P;
    constexpr int PRC = kCluPitch - 1;
    extern __shared__ __align__(16) float sm[];
    __shared__ uint64_t mb[kHaloBars];
    __shared__ int failed;
    __shared__ float acc_src;
    __shared__ uint32_t tmem_slot;
    float *U0 = sm, *U1 = U0 + FS, *K = U1 + FS, *IC = K + RC * P;
    float *ST = IC + a.nr, *RSw = ST + e.chunk * a.nr;
    const int g0 = crank * RC;
    const uint32_t tmem = tmem_alloc(&tmem_slot, kCluTmemCols);
    for (int i = tid; i < 2 * FS; i += nth) sm[i] = 0.f;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    for (int i = tid; i < a.nr; i += nth) {
        const int rz = a.rec_pz[i], rx = a.rec_px[i];
        const float vv = vb[min(rz, a.nz - 1) * a.nx + min(max(rx - a.nb, 0), a.nx - 1)];
        const double vdt = (double)vv * a.dtd;
        IC[i] = (float)(vdt * vdt / (1.0 - e_cell(rx, rz, a)));   // kappa / B
    }
    int bad = 0;
    for (int i = tid; i < RC * P; i += nth) {
        const int lr = i / P, px = i - (i / P) * P, gz = g0 + lr;
        float k = 0.f;
        if (gz < NZ && px < NX) {
            const float vv = vb[min(gz, a.nz - 1) * a.nx + min(max(px - a.nb, 0), a.nx - 1)];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, px, gz, a);
        }
        K[i] = k;
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    __syncthreads();   // the kappa A table is complete before it goes to tensor memory
    // inactive threads (past the last strip) run the row code on strip 0,
    // columns 0 and 1, with every write gated (TMEM accesses are warp-collective)
    const int NXP = NX / 2;
    const int strip = tid / NXP;
    const bool active = strip < e.nstrip;
    const int x = active ? 2 * (tid % NXP) : 0;
    const int l0 = active ? strip * RW : 0;
    const bool has_up = crank > 0, has_dn = crank + 1 < C;
    const bool send_up = active && strip == 0 && has_up;
    const bool send_dn = active && strip == e.nstrip - 1 && has_dn;
    const bool top_strip = active && strip == 0 && crank == 0;
    const unsigned halo_bytes = (unsigned)((has_up ? 1 : 0) + (has_dn ? 1 : 0)) * 8u * NX;
    if (tid == 0) {
        halo_init(mb, halo_bytes, a.nt);
        failed = 0;
        acc_src = 0.f;
    }
    // receivers owned by this thread (one per column of a strip at most)
    int inj0 = -1, inj1 = -1;
    for (int i = 0; i < a.nr; ++i) {
        const int rz = a.rec_pz[i] - g0, rx = a.rec_px[i];
        if (active && rz >= l0 && rz < l0 + RW) {
            if (rx == x) inj0 = i;
            if (rx == x + 1) inj1 = i;
        }
    }
    const int inj0_off = inj0 >= 0 ? (a.rec_pz[inj0] - g0 + 2) * P + x + 2 : 0;
    const int inj1_off = inj1 >= 0 ? (a.rec_pz[inj1] - g0 + 2) * P + x + 3 : 0;
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const bool src_here = sz >= g0 && sz < g0 + RC;
    const int warp = tid >> 5;
    const uint32_t tacc = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                          (uint32_t)(kCluWarpCols * (warp >> 2));
    const uint32_t tkd = tacc + kCluSumCols;
    // imaging sums (zero) and (kappa A, 2A) of the thread's cells into its TMEM lane
    const float zbf = (float)(g0 + l0 - (a.nz - 1));
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        tmem_st2(tacc + 2 * r, make_float2(0.f, 0.f));
        const float ez = ez_of(zbf + (float)r, a);
        const float2 h = f2::add(f2::splat(1.f),
                                 f2::add(make_float2(ex_of(x, a), ex_of(x + 1, a)), f2::splat(ez)));
        tmem_st4(tkd + 4 * r, f2::ld(K + (l0 + r) * P + x),
                 make_float2(__fdividef(2.f, h.x), __fdividef(2.f, h.y)));
    }
    tmem_wait_st();
    const size_t plane = (size_t)C * RC * PRC;
    // this CTA's rows of a record plane (for the L2 prefetch)
    const size_t cta_off = (size_t)g0 * PRC, cta_bytes = (size_t)RC * PRC * 4;
    const float *plane_last = a.snap + ((size_t)bs * a.rec_planes + (a.nt - 1)) * plane;
    const float *sr = plane_last + (size_t)(g0 + l0) * PRC + x;
    float2 rq[kCluKR];
#pragma unroll
    for (int i = 0; i < kCluKR; ++i) rq[i] = f2::ld(sr + i * PRC);
    if (a.nt > 1) prefetch_plane_l2(plane_last - plane + cta_off, cta_bytes, tid);
    cl.sync();   // every CTA's fields are zero and its mbarriers set up

    for (int j0 = 0; j0 < a.nt; j0 += e.chunk) {
        const int nch = min(e.chunk, a.nt - j0);
        const float *ab = a.adj + (size_t)bs * a.nr * a.nt;
        for (int q = tid; q < nch * a.nr; q += nth) {
            const int i = q / nch, jj = q - (q / nch) * nch;
            ST[jj * a.nr + i] = IC[i] * ab[(size_t)i * a.nt + (a.nt - 1 - (j0 + jj))];
        }
        for (int q = tid; q < nch; q += nth) RSw[q] = ricker_scaled(a.nt - 1 - (j0 + q), a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (tid == 0 && j + 3 <= a.nt && !*(volatile int *)&failed)
                halo_arm(&mb[(j + 3) & 3], halo_bytes);
            if (inj0 >= 0) nxt[inj0_off] -= ST[jj * a.nr + inj0];   // (kappa/B) q
            if (inj1 >= 0) nxt[inj1_off] -= ST[jj * a.nr + inj1];
            if (j + 2 < a.nt) prefetch_plane_l2(plane_last - (size_t)(j + 2) * plane + cta_off,
                                                cta_bytes, tid);
            const float *sr_next = (j + 1 < a.nt) ? sr - plane : sr;
            float *np = nxt + (l0 + 2) * P + x + 2;
            adj_rows_pair<P, PRC, RW, kCluKR, TOPBC>(cur + (l0 + 2) * P + x + 2, np, sr, sr_next,
                                                     top_strip, active, tacc, tkd, rq, a);
            tmem_wait_st();
            sr = sr_next;
            // a CTA whose wait ran out sends no more halo rows
            if (active && !e.withhold && !*(volatile int *)&failed)
                send_edges_pair<P, RW>(np, RC, crank, send_up, send_dn, &mb[(j + 1) & 3]);
            __syncthreads();
            if (tid == nth - 1 && src_here)
                acc_src = fmaf(nxt[(sz - g0 + 2) * P + sx + 2], RSw[jj], acc_src);
            halo_wait(&mb[(j + 1) & 3], halo_parity(j + 1), &failed, a.status, e.wait_ns);
        }
        __syncthreads();
    }
    // imaging sums of this CTA's rows and the source-cell sum to the fold
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        uint32_t s0, s1;
        tmem_ld2(tacc + 2 * r, s0, s1);
        tmem_wait_ld();
        const int gz = g0 + l0 + r;
        if (active && gz < NZ) {
            float *dst = e.acc + ((size_t)bs * NZ + gz) * e.NXp + x;
            dst[0] = __uint_as_float(s0);
            dst[1] = __uint_as_float(s1);
        }
    }
    if (tid == 0 && src_here) e.acc_src[bs] = acc_src;
    tmem_free(tmem, kCluTmemCols);
    cl.sync();   // no CTA leaves while a neighbour may still write into it
}

template <typename Kern>
cudaError_t launch_clu(Kern kern, const PropArgs &a, const ClusterArgs &e, int nbs, int threads,
                       size_t smem, cudaStream_t st)
{
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nbs * e.C));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)e.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, e);
}

}  // namespace

size_t cluster_smem(int RC, int P, bool adj, int chunk, int nr, bool pair)
{
    // two levels with halo rows + one per-cell table (+ the imaging sums,
    // which the column-pair adjoint keeps in tensor memory, and kappa/B per
    // receiver for the adjoint) + staging of receiver samples and the wavelet
    const size_t sums = adj && !pair ? (size_t)RC * (P - 1) : 0;
    return ((size_t)2 * (RC + 4) * P + (size_t)RC * P + sums + (adj ? (size_t)nr : 0) +
            (size_t)chunk * (nr + 1)) *
           sizeof(float);
}

cudaError_t launch_cluster(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                           cudaStream_t st, bool wait_check)
{
    const int nbs = pl.p.batch * pl.p.ns;
    ClusterArgs e = pl.clu;
    // the self-check withholds every halo row and bounds each wait by 20 ms
    e.withhold = wait_check ? 1 : 0;
    e.wait_ns = wait_check ? 20000000ull : kHaloWaitNs;
    e.acc = (float *)(ws + pl.ws_t_acc);
    e.acc_src = (float *)(ws + pl.ws_t_accsrc);
    e.chunk = adj ? pl.clu_chunk_adj : pl.clu_chunk_fwd;
    const size_t smem = cluster_smem(e.RC, e.P, adj, e.chunk, pl.p.nr, e.pair != 0);
    const int threads = pl.clu_threads;
    const int tb = pl.p.top_bc;
    const bool store = a.snap != nullptr;
#define FWI_CLU(PP, RSV)                                                                        \
    if (e.P == PP && e.RS == RSV) {                                                             \
        if (adj)                                                                                \
            return tb ? launch_clu(k_clu_adj<PP, RSV, 1>, a, e, nbs, threads, smem, st)         \
                      : launch_clu(k_clu_adj<PP, RSV, 0>, a, e, nbs, threads, smem, st);        \
        if (store)                                                                              \
            return tb ? launch_clu(k_clu_fwd<PP, RSV, 1, true>, a, e, nbs, threads, smem, st)   \
                      : launch_clu(k_clu_fwd<PP, RSV, 0, true>, a, e, nbs, threads, smem, st);  \
        return tb ? launch_clu(k_clu_fwd<PP, RSV, 1, false>, a, e, nbs, threads, smem, st)      \
                  : launch_clu(k_clu_fwd<PP, RSV, 0, false>, a, e, nbs, threads, smem, st);     \
    }
    if (e.pair) {
        if (e.P != kCluPairPitch || e.RS != kCluPairRows) return cudaErrorInvalidValue;
        constexpr int PP = kCluPairPitch, RW = kCluPairRows;
        // the adjoint takes all of its SM's tensor memory: it asks for more
        // than half the SM's shared memory, so no second CTA (whose allocation
        // would wait for this one, or for a CTA of its own cluster) shares the SM
        const size_t smem_adj = smem > kCluSoloSmem ? smem : kCluSoloSmem;
        if (adj)
            return tb ? launch_clu(k_clu_adj_pair<PP, RW, 1>, a, e, nbs, threads, smem_adj, st)
                      : launch_clu(k_clu_adj_pair<PP, RW, 0>, a, e, nbs, threads, smem_adj, st);
        if (store)
            return tb ? launch_clu(k_clu_fwd_pair<PP, RW, 1, true>, a, e, nbs, threads, smem, st)
                      : launch_clu(k_clu_fwd_pair<PP, RW, 0, true>, a, e, nbs, threads, smem, st);
        return tb ? launch_clu(k_clu_fwd_pair<PP, RW, 1, false>, a, e, nbs, threads, smem, st)
                  : launch_clu(k_clu_fwd_pair<PP, RW, 0, false>, a, e, nbs, threads, smem, st);
    }
    FWI_CLU(kCluPitch, 13)
    FWI_CLU(kCluPitch, 19)
#undef FWI_CLU
    return cudaErrorInvalidValue;
}

}  // namespace fwi
