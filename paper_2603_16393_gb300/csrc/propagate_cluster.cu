// propagate_cluster.cu -- propagators for padded grids too large for one
// CTA's shared memory but small enough for a cluster's (for example 256 x 256
// models with a 40-cell layer: 296 x 336 cells).
//
// The grid of a (model, shot) is split by rows across a cluster of kClu CTAs:
// CTA c of the cluster keeps rows [c RC, (c+1) RC) of both time levels in its
// shared memory, with two halo rows above and below.  A thread that computes
// one of the two first (last) rows of its CTA also stores the new value into
// the bottom (top) halo rows of the CTA above (below) through distributed
// shared memory, and one cluster barrier per step (release / acquire) makes
// those stores visible before the next step reads them.  The fields never
// leave the chip; only the wavefield record, traces and gradients go to HBM.
//
// Same recurrences and coefficient formation as the single-CTA resident
// kernels: forward in increment form with a difference Laplacian and the
// FP64-formed A B table; adjoint in the self-adjoint phi = kappa A mu form
// (the receivers' adjoint source through the old level, imaging acc +=
// psi^{j+1} t^{nt-1-j}, source-cell term kept apart), its imaging sums in
// shared memory; they go to the tiled kernels' buffers, whose fold kernel
// finishes.
// The record of a cluster plan has kClusterCTAs RC rows per plane at the row
// pitch P - 1, so that every record access is a compile-time offset.
//
// Every CTA of a cluster executes the same sequence of cluster barriers (no
// early exit: an invalid velocity only sets the status word).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fwi_device.cuh"
#include "fwi_internal.cuh"

namespace cg = cooperative_groups;

namespace fwi {

namespace {

using dev::e_cell;
using dev::ex_of;
using dev::ez_of;
using dev::kappaA_cell;
using dev::ricker_scaled;

// Values moved through an opaque register copy are recomputed where used
// instead of being hoisted out of the time loop.
__device__ __forceinline__ float opaque_c(float x)
{
    float y;
    asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int P, int RS, int TOPBC, bool STORE>
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(clu_max_threads(RS), 1)
k_clu_fwd(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int bs = blockIdx.x / kClusterCTAs, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (e.rows_cap + 4) * P;
    extern __shared__ float sm[];
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
        const int lr = l0 + r, gz = g0 + lr;
        float k = 0.f;
        if (active && lr < RC && gz < NZ) {
            const float vv = vb[min(gz, a.nz - 1) * a.nx + ixc];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            k = kappaA_cell(vv, x, gz, a);
        }
        ka[r] = k;
        vi[r] = 0.f;
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    const bool has_up = crank > 0, has_dn = crank + 1 < kClusterCTAs;
    // source owner
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const int src_row = (active && x == sx && sz >= g0 + l0 && sz < g0 + l0 + RS && sz - g0 < RC)
                            ? sz - g0 - l0 : -1;
    float ka_src = 0.f;
#pragma unroll
    for (int r = 0; r < RS; ++r)
        if (r == src_row) ka_src = ka[r];
    // record plane of step j: rows [0, kClusterCTAs RC) at the compile-time pitch PRC
    constexpr int PRC = P - 1;
    const size_t plane = (size_t)kClusterCTAs * RC * PRC;
    float *sw = STORE ? a.snap + (size_t)bs * a.rec_planes * plane + (size_t)(g0 + l0) * PRC + x : nullptr;
    cl.sync();   // every CTA's fields are zero before any neighbour stores into them

    for (int j0 = 0; j0 < a.nt; j0 += e.chunk) {
        const int nch = min(e.chunk, a.nt - j0);
        for (int q = tid; q < nch; q += nth) RSw[q] = ricker_scaled(j0 + q, a);
        __syncthreads();
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? U1 : U0;
            float *nxt = (j & 1) ? U0 : U1;
            if (active) {
                const float *cp = cur + (l0 + 2) * P + x + 2;
                float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    const int lr = l0 + r;
                    const float *c = cp + r * P;
                    const float wp2 = c[2 * P];
                    const float dzA = (wm1 - w0) + (wp1 - w0);
                    const float dzB = (wm2 - w0) + (wp2 - w0);
                    const float dxA = (c[-1] - w0) + (c[1] - w0);
                    const float dxB = (c[-2] - w0) + (c[2] - w0);
                    float lap = a.cx1 * dxA;
                    lap = fmaf(a.cx2, dxB, lap);
                    lap = fmaf(a.cz1, dzA, lap);
                    lap = fmaf(a.cz2, dzB, lap);
                    if (lr < RC) {
                        const float ab = ABt[lr * P + x];
                        vi[r] = fmaf(ka[r], lap, ab * vi[r]);
                        float un = w0 + vi[r];
                        if (r == src_row) {
                            // point source: + kappa A s (increment and field)
                            const float d = ka_src * RSw[jj];
                            vi[r] += d;
                            un += d;
                        }
                        nxt[(lr + 2) * P + x + 2] = un;
                        // halo rows of the neighbours (their copies of this level)
                        if (lr < 2 && has_up)
                            cl.map_shared_rank(nxt, crank - 1)[(RC + lr + 2) * P + x + 2] = un;
                        if (lr >= RC - 2 && has_dn)
                            cl.map_shared_rank(nxt, crank + 1)[(lr - RC + 2) * P + x + 2] = un;
                        if (TOPBC == 1 && crank == 0 && (lr == 1 || lr == 2))
                            nxt[(2 - lr) * P + x + 2] = un;   // mirrored ghost row -lr
                        if (STORE) sw[r * PRC] = lap;
                    }
                    wm2 = wm1;
                    wm1 = w0;
                    w0 = wp1;
                    wp1 = wp2;
                }
            }
            if (STORE) sw += plane;
            cl.sync();
            for (int i = tid; i < a.nr; i += nth) {
                const int rz = a.rec_pz[i] - g0;
                if (rz >= 0 && rz < RC) ST[jj * a.nr + i] = nxt[(rz + 2) * P + a.rec_px[i] + 2];
            }
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
}

template <int P, int RS, int TOPBC>
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(clu_max_threads(RS), 1)
k_clu_adj(const __grid_constant__ PropArgs a, const __grid_constant__ ClusterArgs e)
{
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int bs = blockIdx.x / kClusterCTAs, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NX = a.NX, NZ = a.NZ, RC = e.RC;
    const int FS = (e.rows_cap + 4) * P;
    extern __shared__ float sm[];
    constexpr int PRC = P - 1;
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
    const bool has_up = crank > 0, has_dn = crank + 1 < kClusterCTAs;
    // receiver owned by this thread (at most one per column of a strip)
    int inj_slot = -1;
    for (int i = 0; i < a.nr; ++i) {
        const int rz = a.rec_pz[i] - g0, rx = a.rec_px[i];
        if (active && x == rx && rz >= l0 && rz < l0 + RS && rz < RC) inj_slot = i;
    }
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const bool src_here = sz >= g0 && sz < g0 + RC;
    __shared__ float acc_src;
    if (tid == 0) acc_src = 0.f;
    const size_t plane = (size_t)kClusterCTAs * RC * PRC;
    float sv[RS];
    // record plane read next: forward step nt-1, then one plane back per step
    const float *sr = a.snap + ((size_t)bs * a.rec_planes + (a.nt - 1)) * plane + (size_t)(g0 + l0) * PRC + x;
#pragma unroll
    for (int r = 0; r < RS; ++r) sv[r] = (active && l0 + r < RC) ? sr[r * PRC] : 0.f;
    float *ac = ACC + l0 * PRC + x;
    cl.sync();

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
            if (inj_slot >= 0) {
                const int rz = a.rec_pz[inj_slot] - g0, rx = a.rec_px[inj_slot];
                nxt[(rz + 2) * P + rx + 2] -= ST[jj * a.nr + inj_slot];   // (kappa/B) q
            }
            if (j + 1 < a.nt) sr -= plane;
            if (active) {
                const float *cp = cur + (l0 + 2) * P + x + 2;
                float *np = nxt + (l0 + 2) * P + x + 2;
                const float exs = opaque_c(ex), zb = opaque_c(zbf);
                float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
#pragma unroll
                for (int r = 0; r < RS; ++r) {
                    const int lr = l0 + r;
                    const float *c = cp + r * P;
                    const float wp2 = c[2 * P];
                    float lap = a.c0 * w0;
                    lap = fmaf(a.cx1, c[-1] + c[1], lap);
                    lap = fmaf(a.cx2, c[-2] + c[2], lap);
                    lap = fmaf(a.cz1, wm1 + wp1, lap);
                    lap = fmaf(a.cz2, wm2 + wp2, lap);
                    if (TOPBC == 1 && crank == 0 && (lr == 1 || lr == 2))
                        // transpose of the mirrored top: reflected weights onto rows 1, 2
                        lap += (lr == 1) ? a.cz1 * wm1 + a.cz2 * w0 : a.cz2 * wm2;
                    if (lr < RC) {
                        const float ee = exs + ez_of(zb + (float)r, a);
                        const float A2 = __fdividef(2.f, 1.f + ee);   // 2A
                        const float AB = A2 - 1.f;                     // A B
                        const float fo = np[r * P];
                        const float fn = fmaf(K[lr * P + x], lap, fmaf(A2, w0, -AB * fo));
                        np[r * P] = fn;
                        if (lr < 2 && has_up)
                            cl.map_shared_rank(nxt, crank - 1)[(RC + lr + 2) * P + x + 2] = fn;
                        if (lr >= RC - 2 && has_dn)
                            cl.map_shared_rank(nxt, crank + 1)[(lr - RC + 2) * P + x + 2] = fn;
                        ac[r * PRC] = fmaf(fn, sv[r], ac[r * PRC]);
                        sv[r] = sr[r * PRC];
                    }
                    wm2 = wm1;
                    wm1 = w0;
                    w0 = wp1;
                    wp1 = wp2;
                }
            }
            cl.sync();
            if (tid == nth - 1 && src_here)
                acc_src = fmaf(nxt[(sz - g0 + 2) * P + sx + 2], RSw[jj], acc_src);
        }
        __syncthreads();
    }
    // imaging sums of this CTA's rows and the source-cell sum to the fold
    for (int i = tid; i < RC * NX; i += nth) {
        const int lr = i / NX, px = i - (i / NX) * NX, gz = g0 + lr;
        if (gz < NZ) e.acc[((size_t)bs * NZ + gz) * e.NXp + px] = ACC[lr * PRC + px];
    }
    if (tid == 0 && src_here) e.acc_src[bs] = acc_src;
}

template <typename Kern>
cudaError_t launch_clu(Kern kern, const PropArgs &a, const ClusterArgs &e, int nbs, int threads,
                       size_t smem, cudaStream_t st)
{
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<nbs * kClusterCTAs, threads, smem, st>>>(a, e);
    return cudaGetLastError();
}

}  // namespace

size_t cluster_smem(int rows_cap, int RC, int P, bool adj, int chunk, int nr)
{
    // two levels with halo rows + one per-cell table (+ the imaging sums and
    // kappa/B per receiver for the adjoint) + staging of receiver samples and
    // the wavelet
    return ((size_t)2 * (rows_cap + 4) * P + (size_t)RC * P +
            (adj ? (size_t)RC * (P - 1) + nr : 0) + (size_t)chunk * (nr + 1)) * sizeof(float);
}

cudaError_t launch_cluster(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                           cudaStream_t st)
{
    const int nbs = pl.p.batch * pl.p.ns;
    ClusterArgs e = pl.clu;
    e.acc = (float *)(ws + pl.ws_t_acc);
    e.acc_src = (float *)(ws + pl.ws_t_accsrc);
    e.chunk = adj ? pl.clu_chunk_adj : pl.clu_chunk_fwd;
    const size_t smem = cluster_smem(e.rows_cap, e.RC, e.P, adj, e.chunk, pl.p.nr);
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
    FWI_CLU(kCluPitch, 13)
    FWI_CLU(kCluPitch, 19)
#undef FWI_CLU
    return cudaErrorInvalidValue;
}

}  // namespace fwi
