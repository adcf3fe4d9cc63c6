// propagate.cu -- shared-memory-resident acoustic propagator for sm_103a.
//
// Forward (Eq. 1, Sec. 2.1 / 6.1):
//   u^{j+1} = A (2 u^j - B u^{j-1} + kappa (L u^j + s^j)),  j = 0..nt-1
//   kappa = v_pad^2 dt^2,  A = 1/(1+e), B = 1-e, e = eta dt/2,
//   s^j = f(j dt)/(dx dz) at the source cell (Ricker, Sec. 6.1),
//   d[r][j] = u^{j+1} at receiver r; the snapshot of step j is t^j = L u^j + s^j.
//
// Adjoint.  With mu the discrete adjoint of u and phi = kappa A mu, the
// transposed recurrence becomes the same propagator run on reversed time:
//   psi^{j+1} = A (2 psi^j - B psi^{j-1} + kappa (L^T psi^j + R^T r^{nt-1-j}))
// with psi^j = phi^{nt+1-j}; the imaging condition is
//   dJ/dv_pad = (2 / v_pad) sum_j psi^{j+1} t^{nt-1-j}.
// L is symmetric with zero ghosts; with the mirrored top (top_bc = 1) the
// transpose adds the reflected weights back onto rows 1 and 2.
//
// Layout: one CTA per (model, shot) holds both time levels of the padded
// field (with a two-cell ghost ring) and kappa in shared memory for the whole
// time loop; thread t owns a column strip of `rows` cells at one padded
// column, keeps a 5-value z window in registers and reads its x neighbours
// from shared memory.  One barrier per time step.
#include <cuda_runtime.h>

#include <cmath>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr float kPi = 3.14159265358979323846f;

// Returns x through an opaque move: values derived from it inside the time
// loop are recomputed every step instead of being hoisted out of the loop
// (per-row damping coefficients would pin two registers per row).
__device__ __forceinline__ float opaque_g(float x)
{
    float y;
    asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int MAXROWS, bool ADJ, int TOPBC>
__global__ void __launch_bounds__(ADJ ? kMaxThreadsAdj : kMaxThreadsFwd, 1)
k_propagate(const __grid_constant__ PropArgs a)
{
    extern __shared__ float sm[];
    const int NX = a.NX, NZ = a.NZ;
    const int P = NX + 4;
    const int fsz = (NZ + 4) * P;
    float *F0 = sm;
    float *F1 = sm + fsz;
    float *K = sm + 2 * fsz;
    float *ST = K + NZ * NX;
    const int bs = blockIdx.x;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int tid = threadIdx.x, nth = blockDim.x;

    for (int i = tid; i < 2 * fsz; i += nth) sm[i] = 0.f;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    int bad = 0;
    for (int i = tid; i < NZ * NX; i += nth) {
        const int pz = i / NX, px = i - (i / NX) * NX;
        const int iz = min(pz, a.nz - 1);
        const int ix = min(max(px - a.nb, 0), a.nx - 1);
        const float vv = vb[iz * a.nx + ix];
        if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
        const double vdt = (double)vv * a.dtd;
        K[i] = (float)(vdt * vdt);
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
        return;
    }

    const int x = tid % NX, strip = tid / NX;
    const bool active = strip < a.nstrip;
    const int z0 = strip * a.rows;
    const int myrows = active ? max(0, min(a.rows, NZ - z0)) : 0;

    // damping: e = ex(x) + ez(z); rows above the bottom layer use constants
    float cxd = 0.f;
    if (x < a.nb) cxd = (float)(a.nb - x);
    else if (x > a.nb + a.nx - 1) cxd = (float)(x - (a.nb + a.nx - 1));
    const float ex = a.ex0 * (cxd * a.inv_nb) * (cxd * a.inv_nb);
    const double exd = a.ex0d * ((double)cxd / a.nb) * ((double)cxd / a.nb);
    const float A0 = (float)(1.0 / (1.0 + exd)), B0 = (float)(1.0 - exd);

    // point injection owned by this thread (host guarantees at most one)
    int inj_row = -1, inj_slot = -1;
    if (!ADJ) {
        const int sz = a.src_pz[s], sx = a.src_px[s];
        if (myrows > 0 && x == sx && sz >= z0 && sz < z0 + myrows) inj_row = sz - z0;
    } else {
        for (int i = 0; i < a.nr; ++i) {
            const int rz = a.rec_pz[i], rx = a.rec_px[i];
            if (myrows > 0 && x == rx && rz >= z0 && rz < z0 + myrows) {
                inj_row = rz - z0;
                inj_slot = i;
            }
        }
    }

    const size_t plane = (size_t)NZ * NX;
    float *snap_bs = a.snap ? a.snap + (size_t)bs * a.rec_planes * plane : nullptr;
    const int cell0 = z0 * NX + x;
    const float *kp = K + cell0;
    const int jb = a.j_begin, je = a.j_end;

    float acc[ADJ ? MAXROWS : 1];
    float sv[ADJ ? MAXROWS : 1];
    if (ADJ) {
        const float *s0 = snap_bs + (size_t)(a.nt - 1 - jb - a.rec_base) * plane + cell0;
#pragma unroll
        for (int r = 0; r < MAXROWS; ++r) {
            acc[r] = 0.f;
            sv[r] = (r < myrows) ? s0[r * NX] : 0.f;
        }
    }
    // resume at step jb: levels j and j-1 (the adjoint also its imaging sums)
    const float *rs = ADJ ? (jb > 0 ? a.astate + (size_t)bs * 3 * plane : nullptr)
                          : (a.resume ? a.resume + (size_t)bs * 2 * plane : nullptr);
    if (rs) {
        // flat copy of both levels (per-owner copies cost registers in the
        // time loop), then the owner's imaging sums
        float *cur = (jb & 1) ? F1 : F0, *old = (jb & 1) ? F0 : F1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            cur[(z + 2) * P + xx + 2] = rs[i];
            old[(z + 2) * P + xx + 2] = rs[plane + i];
            if (!ADJ && TOPBC == 1 && (z == 1 || z == 2))
                cur[(2 - z) * P + xx + 2] = rs[i];   // mirrored ghost row -z
        }
        if (ADJ) {
#pragma unroll
            for (int r = 0; r < MAXROWS; ++r)
                if (r < myrows) acc[r] = rs[2 * plane + (z0 + r) * NX + x];
        }
    }
    __syncthreads();

    for (int j0 = jb, nch = 0; j0 < je; j0 += nch) {
        nch = min(a.chunk, je - j0);
        if (!ADJ && a.ckpt) {
            // chunks end at checkpoint steps; the state at the first step of
            // a chunk that is one is saved here (both levels, flat copy)
            nch = min(nch, (j0 / a.ckpt_every + 1) * a.ckpt_every - j0);
            if (j0 % a.ckpt_every == 0) {
                const float *cur = (j0 & 1) ? F1 : F0, *old = (j0 & 1) ? F0 : F1;
                float *cs = a.ckpt + ((size_t)(j0 / a.ckpt_every) * gridDim.x + bs) * 2 * plane;
                for (int i = tid; i < NZ * NX; i += nth) {
                    const int z = i / NX, xx = i - (i / NX) * NX;
                    cs[i] = cur[(z + 2) * P + xx + 2];
                    cs[plane + i] = old[(z + 2) * P + xx + 2];
                }
            }
        }
        if (ADJ) {
            const float *ab = a.adj + (size_t)bs * a.nr * a.nt;
            for (int e = tid; e < nch * a.nr; e += nth) {
                const int i = e / nch, jj = e - (e / nch) * nch;
                ST[jj * a.nr + i] = ab[(size_t)i * a.nt + (a.nt - 1 - (j0 + jj))];
            }
            __syncthreads();
        }
        for (int jj = 0; jj < nch; ++jj) {
            const int j = j0 + jj;
            const float *cur = (j & 1) ? F1 : F0;
            float *old = (j & 1) ? F0 : F1;

            float inj = 0.f;
            if (inj_row >= 0) {
                if (!ADJ) {
                    const float t = (float)((double)j * a.dtd - a.t0d);
                    const float q = (kPi * a.fp * t) * (kPi * a.fp * t);
                    inj = a.src_scale * (1.f - 2.f * q) * expf(-q);
                } else {
                    inj = ST[jj * a.nr + inj_slot];
                }
            }

            const float exs = opaque_g(ex);
            if (myrows > 0) {
                const float *cp = cur + (z0 + 2) * P + x + 2;
                float *op = old + (z0 + 2) * P + x + 2;
                float *row0 = old + 2 * P + x + 2;
                float *snap_w = (!ADJ && snap_bs)
                                    ? snap_bs + (size_t)(j - a.rec_base) * plane + cell0 : nullptr;
                const bool pf = ADJ && (j + 1 < je);
                const float *snap_r =
                    pf ? snap_bs + (size_t)(a.nt - 2 - j - a.rec_base) * plane + cell0 : nullptr;
                float wm2 = cp[-2 * P], wm1 = cp[-P], w0 = cp[0], wp1 = cp[P];
#pragma unroll
                for (int r = 0; r < MAXROWS; ++r) {
                    if (r < myrows) {
                        const float *c = cp + r * P;
                        const float wp2 = c[2 * P];
                        float lap = a.c0 * w0 + a.cx1 * (c[-1] + c[1]) + a.cx2 * (c[-2] + c[2]) +
                                    a.cz1 * (wm1 + wp1) + a.cz2 * (wm2 + wp2);
                        const int z = z0 + r;
                        if (ADJ && TOPBC == 1) {
                            if (z == 1) lap += a.cz1 * wm1 + a.cz2 * w0;
                            if (z == 2) lap += a.cz2 * wm2;
                        }
                        if (r == inj_row) lap += inj;
                        float A = A0, B = B0;
                        if (z >= a.nz) {
                            const float cz = (float)(z - (a.nz - 1)) * a.inv_nb;
                            const float e = exs + a.ez0 * cz * cz;
                            A = 1.f / (1.f + e);
                            B = 1.f - e;
                        }
                        const float fo = op[r * P];
                        const float fn = A * (fmaf(kp[r * NX], lap, 2.f * w0) - B * fo);
                        op[r * P] = fn;
                        if (!ADJ && TOPBC == 1) {
                            if (z == 1) row0[-P] = fn;
                            if (z == 2) row0[-2 * P] = fn;
                        }
                        if (!ADJ && snap_w) snap_w[r * NX] = lap;
                        if (ADJ) {
                            acc[r] = fmaf(fn, sv[r], acc[r]);
                            if (pf) sv[r] = snap_r[r * NX];
                        }
                        wm2 = wm1;
                        wm1 = w0;
                        w0 = wp1;
                        wp1 = wp2;
                    }
                }
            }
            __syncthreads();
            if (!ADJ && tid < a.nr)
                ST[jj * a.nr + tid] = old[(a.rec_pz[tid] + 2) * P + a.rec_px[tid] + 2];
        }
        if (!ADJ) {
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

    if (ADJ && je < a.nt) {
        // suspend: levels psi^je, psi^(je-1) and the imaging sums
        __syncthreads();
        float *st = a.astate + (size_t)bs * 3 * plane;
        const float *cur = (je & 1) ? F1 : F0, *old = (je & 1) ? F0 : F1;
        for (int i = tid; i < NZ * NX; i += nth) {
            const int z = i / NX, xx = i - (i / NX) * NX;
            st[i] = cur[(z + 2) * P + xx + 2];
            st[plane + i] = old[(z + 2) * P + xx + 2];
        }
#pragma unroll
        for (int r = 0; r < MAXROWS; ++r)
            if (r < myrows) st[2 * plane + (z0 + r) * NX + x] = acc[r];
        return;
    }

    if (ADJ) {
        // dJ/dv_pad = 2 acc / v_pad, then fold the absorbing layer onto the
        // physical edge cells (transpose of the edge replication), columns
        // first, then rows, each in a fixed order.
        __syncthreads();
        float *G = F0;            // [NZ][NX]
        float *T = F1;            // [NZ][nx]
#pragma unroll
        for (int r = 0; r < MAXROWS; ++r) {
            if (r < myrows) {
                const int z = z0 + r;
                const int iz = min(z, a.nz - 1);
                const int ix = min(max(x - a.nb, 0), a.nx - 1);
                const float vp = vb[iz * a.nx + ix];
                G[z * NX + x] = 2.f * acc[r] / vp;
            }
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
}

}  // namespace

// grad[b][i] = sum_s gshot[b][s][i], s in increasing order.
__global__ void k_shot_sum(int B, int ns, int n, const float *__restrict__ gshot,
                           float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= n || b >= B) return;
    const float *g = gshot + (size_t)b * ns * n + i;
    float sum = 0.f;
    for (int s = 0; s < ns; ++s) sum += g[(size_t)s * n];
    grad[(size_t)b * n + i] = sum;
}

PropArgs make_args(const Plan &pl)
{
    const fwi_problem &p = pl.p;
    PropArgs a{};
    a.nz = p.nz; a.nx = p.nx; a.nb = p.nb; a.NZ = pl.NZ; a.NX = pl.NX;
    a.nt = p.nt; a.ns = p.ns; a.nr = p.nr;
    a.nzs = pl.nzs;
    a.units = p.batch * p.ns;
    a.dt = (float)p.dt;
    const double ix2 = 1.0 / ((double)p.dx * p.dx), iz2 = 1.0 / ((double)p.dz * p.dz);
    a.c0 = (float)(-2.5 * (ix2 + iz2));
    a.cx1 = (float)(4.0 / 3.0 * ix2);
    a.cx2 = (float)(-1.0 / 12.0 * ix2);
    a.cz1 = (float)(4.0 / 3.0 * iz2);
    a.cz2 = (float)(-1.0 / 12.0 * iz2);
    {
        const float w[5] = {a.c0, a.cx1, a.cx2, a.cz1, a.cz2};
        for (int k = 0; k < 5; ++k) a.w2[k] = make_float2(w[k], w[k]);
    }
    const double lnR = std::log(1.0 / (double)p.refl_R);
    const double eta0x = p.nb > 0 ? 3.0 * p.v_ref * lnR / (p.nb * (double)p.dx) : 0.0;
    const double eta0z = p.nb > 0 ? 3.0 * p.v_ref * lnR / (p.nb * (double)p.dz) : 0.0;
    a.ex0 = (float)(eta0x * p.dt / 2.0);
    a.ez0 = (float)(eta0z * p.dt / 2.0);
    a.ex0d = eta0x * (double)p.dt / 2.0;
    a.ez0d = eta0z * (double)p.dt / 2.0;
    a.dtd = (double)p.dt;
    a.t0d = (double)pl.t0;
    a.inv_nb = p.nb > 0 ? (float)(1.0 / p.nb) : 0.f;
    a.fp = (float)p.f_peak;
    a.t0 = (float)pl.t0;
    a.src_scale = (float)(1.0 / ((double)p.dx * p.dz));
    a.vmax = (float)p.v_max;
    for (int i = 0; i < p.ns; ++i) {
        a.src_pz[i] = (int16_t)pl.src_pz[i];
        a.src_px[i] = (int16_t)pl.src_px[i];
    }
    for (int i = 0; i < p.nr; ++i) {
        a.rec_pz[i] = (int16_t)pl.rec_pz[i];
        a.rec_px[i] = (int16_t)pl.rec_px[i];
    }
    return a;
}

namespace {


template <int MR, bool ADJ, int TBC>
cudaError_t launch_one(const PropArgs &a, const ResidentShape &sh, int nblocks, cudaStream_t st)
{
    auto kern = k_propagate<MR, ADJ, TBC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh.smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, sh.threads, sh.smem, st>>>(a);
    return cudaGetLastError();
}

template <bool ADJ>
cudaError_t dispatch(PropArgs &a, const Plan &pl, cudaStream_t st)
{
    const int nb = pl.p.batch * pl.p.ns;
    const int tb = pl.p.top_bc;
    const ResidentShape &sh = ADJ ? pl.shape_adj : pl.shape;
    a.rows = sh.rows;
    a.nstrip = sh.nstrip;
    a.chunk = sh.chunk;
    switch (sh.maxrows) {
#define FWI_CASE(MR)                                                              \
    case MR:                                                                      \
        return tb ? launch_one<MR, ADJ, 1>(a, sh, nb, st)                        \
                  : launch_one<MR, ADJ, 0>(a, sh, nb, st);
        FWI_CASE(4)
        FWI_CASE(8)
        FWI_CASE(12)
        FWI_CASE(16)
        FWI_CASE(20)
        FWI_CASE(22)
        FWI_CASE(24)
#undef FWI_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace

bool choose_resident_shape(int NZ, int NX, int nr, bool adj, ResidentShape *out)
{
    const int maxthreads = adj ? kMaxThreadsAdj : kMaxThreadsFwd;
    if (NX > maxthreads || NZ < 1 || NX < 1) return false;
    int nstrip = maxthreads / NX;
    if (nstrip > NZ) nstrip = NZ;
    int rows = (NZ + nstrip - 1) / nstrip;
    nstrip = (NZ + rows - 1) / rows;
    static const int buckets[] = {4, 8, 12, 16, 20, 22, 24};
    int maxrows = 0;
    for (int bkt : buckets)
        if (rows <= bkt) { maxrows = bkt; break; }
    if (maxrows == 0) return false;
    const int threads = ((NX * nstrip + 31) / 32) * 32;
    if (threads > maxthreads) return false;
    const size_t limit = 227 * 1024;
    const size_t fixed = (2 * (size_t)(NZ + 4) * (NX + 4) + (size_t)NZ * NX) * sizeof(float);
    if (fixed + (size_t)nr * sizeof(float) > limit) return false;
    int chunk = (int)((limit - fixed) / ((size_t)nr * sizeof(float)));
    if (chunk > 32) chunk = 32;
    if (chunk < 1) return false;
    out->threads = threads;
    out->nstrip = nstrip;
    out->rows = rows;
    out->maxrows = maxrows;
    out->chunk = chunk;
    out->smem = fixed + (size_t)chunk * nr * sizeof(float);
    return true;
}

namespace {

void apply_window(PropArgs &a, const Window &w)
{
    a.j_begin = w.j_begin;
    a.j_end = w.j_end < 0 ? a.nt : w.j_end;
    a.rec_base = w.rec_base;
    a.rec_planes = w.rec_planes < 0 ? a.nt : w.rec_planes;
    a.resume = w.resume;
    a.ckpt = w.ckpt;
    a.ckpt_every = w.ckpt_every;
    a.astate = w.astate;
    a.asrc = w.asrc;
}

}  // namespace

cudaError_t launch_forward(const Plan &pl, const float *v, float *d_syn, float *snap,
                           void *workspace, cudaStream_t st, const Window &w)
{
    PropArgs a = make_args(pl);
    a.v = v;
    a.d_syn = d_syn;
    a.snap = snap;
    a.status = static_cast<int *>(workspace);
    apply_window(a, w);
    if (pl.cpml) return launch_cpml(pl, false, a, static_cast<unsigned char *>(workspace), st);
    if (pl.cluster)
        return launch_cluster(pl, false, a, static_cast<unsigned char *>(workspace), st,
                              w.wait_check);
    if (pl.tiled)
        return launch_tiled(pl, false, a, static_cast<unsigned char *>(workspace), st,
                            w.wait_check);
    if (pl.fast) {
        a.rows = pl.shape.rows;
        a.nstrip = pl.shape.nstrip;
        a.chunk = pl.shape.chunk;
        return launch_fast(pl, false, a, st);
    }
    return dispatch<false>(a, pl, st);
}

cudaError_t launch_adjoint(const Plan &pl, const float *v, const float *adj, const float *snap,
                           float *grad, float *gshot, void *workspace, cudaStream_t st,
                           const Window &w)
{
    PropArgs a = make_args(pl);
    a.v = v;
    a.adj = adj;
    a.snap = const_cast<float *>(snap);
    a.gshot = gshot;
    a.status = static_cast<int *>(workspace);
    apply_window(a, w);
    cudaError_t e;
    if (pl.cpml) {
        e = launch_cpml(pl, true, a, static_cast<unsigned char *>(workspace), st);
    } else if (pl.cluster) {
        e = launch_cluster(pl, true, a, static_cast<unsigned char *>(workspace), st);
        if (e == cudaSuccess)
            e = launch_tile_fold(pl, a, static_cast<unsigned char *>(workspace), st);
    } else if (pl.tiled) {
        e = launch_tiled(pl, true, a, static_cast<unsigned char *>(workspace), st);
    } else if (pl.fast) {
        a.rows = pl.shape_adj.rows;
        a.nstrip = pl.shape_adj.nstrip;
        a.chunk = pl.shape_adj.chunk;
        e = launch_fast(pl, true, a, st);
    } else {
        e = dispatch<true>(a, pl, st);
    }
    if (e != cudaSuccess) return e;
    if (a.j_end < a.nt || !grad) return cudaSuccess;
    const int n = pl.p.nz * pl.p.nx;
    dim3 grid((n + 255) / 256, pl.p.batch);
    k_shot_sum<<<grid, 256, 0, st>>>(pl.p.batch, pl.p.ns, n, gshot, grad);
    return cudaGetLastError();
}

}  // namespace fwi
