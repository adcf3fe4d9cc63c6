// propagate_tiled.cu -- propagators for padded grids larger than one CTA's
// shared memory (for example 256 x 256 or 512 x 1024 models with a 40-cell
// absorbing layer), same recurrences as the shared-memory resident kernels:
//
//   forward  v^{j+1/2} = A B v^{j-1/2} + kappa A (L u^j + s^j),  u^{j+1} = u^j + v^{j+1/2}
//            (Eq. 1 in increment form, Laplacian on neighbour differences)
//   adjoint  w^{j+1/2} = A B w^{j-1/2} + kappa A (L^T psi^j + q^j),  psi^{j+1} = psi^j + w^{j+1/2}
//            (the same form with L^T; q the receivers' adjoint source), imaging
//            dJ/dv_pad = (2 / v_pad) sum_j psi^{j+1} t^{nt-1-j}
//
// The fields of every (model, shot) live in global memory, [bs][NZ][NXp]
// with NXp = NX rounded up to a multiple of 4 (16-byte rows; the pad columns
// stay zero).  One launch advances all (model, shot) pairs by one time step.
// A CTA owns a 32 x 64 tile.  By default a thread owns four adjacent columns
// and two rows and moves them with 16-byte (float4) loads and stores (the
// column quads below); the scalar shapes give thread (tx, g) column x0 + tx
// and rows z0 + 8g .. z0 + 8g + 7 (or 4 rows).  Either keeps a z window in
// registers, with the same operations per cell, so the same bits.  The current
// level's halo tile (36 x 72 cells; it starts at x0 - 4 so that the copy
// starts on a 16-byte boundary) is moved into shared memory by one
// cp.async.bulk.tensor load completing on an mbarrier; the tensor's
// out-of-bounds fill supplies the zero ghosts around the padded grid (the
// mirrored top rows are copied in after the load).  The per-cell operands
// that have no halo (increment or old level, coefficients, record, imaging
// sums) are read with coalesced loads while the copy is in flight.
//
// Data samples: the launch of step j records d[:, j-1] = u^j from its tile;
// a final gather records d[:, nt-1].
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "fwi_device.cuh"
#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int TX = 64, TZ = 32;
// rows a thread owns (a template bucket the plan's shape picks: 8 -> 256
// threads a CTA, 4 -> 512); a CTA always covers one TZ x TX tile
template <int TRW> __host__ __device__ constexpr int tile_threads() { return TX * TZ / TRW; }
// halo tile: x from x0 - 4 (16-byte aligned start, covers a radius up to 4),
// z from z0 - R for a stencil of radius R (2: 4th order, 4: 8th order)
constexpr int HX = TX + 8;
template <int R> __host__ __device__ constexpr int halo_rows() { return TZ + 2 * R; }
constexpr long kWaitLimit = 1L << 22;                 // mbarrier polls before giving up

// Compact per-launch arguments (one launch per time step).
struct TileArgs {
    int nz, nx, nb, NZ, NX, NXp, nt, ns, nr;
    int j;                      // time step of this launch
    int rec_base;               // record plane of forward step f is f - rec_base
    long long rec_planes;       // record planes per (model, shot)
    int ckpt_every;
    int rzmin, rzmax;           // rows that hold receivers
    double dtd, t0d, ex0d, ez0d;
    float c0, cx1, cx2, cz1, cz2, ex0, ez0, inv_nb, fp, src_scale;
    float cxm[4], czm[4];       // second-difference weights / h^2 for offsets 1..R
    const float *ka, *ab;       // [B][NZ][NXp]: kappa A, A B
    const int *rec;             // [nr]: pz << 16 | px
    const int *src;             // [ns]: pz << 16 | px
    // forward
    float *unext, *vinc;        // u^{j+1} (written), increment (in place)
    float *rec_out;             // record [bs][rec_planes][NZ][NXp], null: off
    float *d_syn;               // [bs][nr][nt], null: off
    float *ckpt;                // checkpoint slots [slot][bs][2][NZ][NX], null: off
    // adjoint (reuses unext = psi^{j+1}, vinc = its increment)
    float *acc, *acc_src;       // imaging sums [bs][NZ][NXp], source-cell sums [bs]
    const float *adj;           // adjoint source [bs][nr][nt]
    const float *rec_in;        // record read by the adjoint
    int *status;
    int withhold;               // 1: load no halo tile (the bounded-wait self-check)
    long long wait_polls;       // bound of one tile wait, in mbarrier polls
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Starts the halo-tile copy (one thread) after arming the mbarrier.
__device__ __forceinline__ void tile_load(float *tile, uint64_t *mbar, const CUtensorMap *tm,
                                         int x, int z, int bs, unsigned bytes)
{
    const unsigned mb = smem_u32(mbar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(z), "r"(bs), "r"(mb)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *mbar)
{
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(mbar))
        : "memory");
    return done != 0;
}

// Every thread waits for the tile (bounded).  Returns false for the whole
// CTA if the copy did not land in time: the status word then holds
// FWI_ERR_DEVICE_TIMEOUT, and the CTA waits once more (bounded) so that no
// copy is left writing into its shared memory when it exits.
__device__ __forceinline__ bool tile_wait(uint64_t *mbar, int *status, long long polls)
{
    bool done = false;
    for (long long it = 0; it < polls && !done; ++it) done = mbar_try(mbar);
    if (__syncthreads_and(done)) return true;
    if (threadIdx.x == 0) set_status(status, FWI_ERR_DEVICE_TIMEOUT);
    for (long long it = 0; it < polls && !done; ++it) done = mbar_try(mbar);
    return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ------------------------------------------------------------------ set-up
// Per-model tables (kappa A, A B) formed in double exactly as the resident
// kernels form them, the receiver and source tables, and the velocity check.
__global__ void __launch_bounds__(256) k_tile_setup(const __grid_constant__ PropArgs a, int NXp,
                                                    float *__restrict__ ka,
                                                    float *__restrict__ ab, int *__restrict__ rec,
                                                    int *__restrict__ src)
{
    const int b = blockIdx.y;
    const float *vb = a.v + (size_t)b * a.nz * a.nx;
    const size_t plane = (size_t)a.NZ * NXp;
    int bad = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int pz = (int)(i / NXp), px = (int)(i - (i / NXp) * NXp);
        float k = 0.f, m = 0.f;
        if (px < a.NX) {
            const float vv = vb[min(pz, a.nz - 1) * a.nx + min(max(px - a.nb, 0), a.nx - 1)];
            if (!(vv > 0.f && vv <= a.vmax)) bad = 1;
            const double e = dev::e_cell(px, pz, a);
            k = dev::kappaA_cell(vv, px, pz, a);
            m = (float)((1.0 - e) / (1.0 + e));
        }
        ka[(size_t)b * plane + i] = k;
        ab[(size_t)b * plane + i] = m;
    }
    if (bad) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    if (blockIdx.x == 0 && b == 0) {
        for (int i = threadIdx.x; i < a.nr; i += blockDim.x)
            rec[i] = ((int)a.rec_pz[i] << 16) | a.rec_px[i];
        for (int i = threadIdx.x; i < a.ns; i += blockDim.x)
            src[i] = ((int)a.src_pz[i] << 16) | a.src_px[i];
    }
}

// ------------------------------------------------------------------ forward step
template <int R, int TOPBC, bool STORE, int TRW>
__global__ void __launch_bounds__(tile_threads<TRW>()) k_tile_fwd(const __grid_constant__ CUtensorMap tm,
                                                       const __grid_constant__ TileArgs a)
{
    constexpr int HZ = halo_rows<R>();
    __shared__ __align__(128) float tile[HZ * HX];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x, tx = tid % TX, g = tid / TX;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, bs = blockIdx.z;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    if (tid == 0) mbar_init(&mbar);
    __syncthreads();
    if (tid == 0 && !a.withhold) tile_load(tile, &mbar, &tm, x0 - 4, z0 - R, bs, HZ * HX * sizeof(float));

    const int x = x0 + tx, zr = z0 + g * TRW;
    const bool colok = x < a.NX;
    const size_t plane = (size_t)a.NZ * a.NXp;
    const float *kab = a.ka + (size_t)b * plane, *abb = a.ab + (size_t)b * plane;
    float *vb = a.vinc + (size_t)bs * plane;
    float ka[TRW], ab[TRW], vi[TRW];
#pragma unroll
    for (int r = 0; r < TRW; ++r) {
        const int z = zr + r;
        const bool ok = colok && z < a.NZ;
        const size_t i = (size_t)z * a.NXp + x;
        ka[r] = ok ? kab[i] : 0.f;
        ab[r] = ok ? abb[i] : 0.f;
        vi[r] = ok ? vb[i] : 0.f;
    }
    if (!tile_wait(&mbar, a.status, a.wait_polls)) return;
    if (TOPBC == 1 && z0 == 0) {
        // mirrored ghost rows: row -k = row k, k = 1..R
        for (int c = tid; c < HX; c += tile_threads<TRW>()) {
#pragma unroll
            for (int k = 1; k <= R; ++k) tile[(R - k) * HX + c] = tile[(R + k) * HX + c];
        }
        __syncthreads();
    }
    // data sample of the previous step at the receivers inside this tile
    if (a.d_syn && a.j > 0 && z0 <= a.rzmax && z0 + TZ > a.rzmin) {
        for (int r = tid; r < a.nr; r += tile_threads<TRW>()) {
            const int pz = a.rec[r] >> 16, px = a.rec[r] & 0xffff;
            if (pz >= z0 && pz < z0 + TZ && px >= x0 && px < x0 + TX)
                a.d_syn[((size_t)bs * a.nr + r) * a.nt + a.j - 1] =
                    tile[(pz - z0 + R) * HX + px - x0 + 4];
        }
    }
    // checkpoint of the state at step j (field u^j, increment v^(j-1/2))
    if (a.ckpt && a.j % a.ckpt_every == 0) {
        const size_t cells = (size_t)a.NZ * a.NX;
        float *st = a.ckpt + ((size_t)(a.j / a.ckpt_every) * gridDim.z + bs) * 2 * cells;
#pragma unroll
        for (int r = 0; r < TRW; ++r) {
            const int z = zr + r;
            if (colok && z < a.NZ) {
                st[(size_t)z * a.NX + x] = tile[(z - z0 + R) * HX + tx + 4];
                st[cells + (size_t)z * a.NX + x] = vi[r];
            }
        }
    }

    const int sp = a.src[s], sz = sp >> 16, sx = sp & 0xffff;
    float *ub = a.unext + (size_t)bs * plane;
    float *rb = STORE ? a.rec_out + ((size_t)bs * a.rec_planes + (a.j - a.rec_base)) * plane
                      : nullptr;
    const float *cp = tile + (g * TRW + R) * HX + tx + 4;
    float w[2 * R + 1];     // z window: w[R + k] = row z + k
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) w[k] = cp[(k - R) * HX];
#pragma unroll
    for (int r = 0; r < TRW; ++r) {
        const float *c = cp + r * HX;
        w[2 * R] = c[R * HX];
        const float w0 = w[R];
        // Laplacian on neighbour differences: sum_m c_m ((u_{-m} - u_0) + (u_{+m} - u_0))
        float lap = a.cxm[0] * ((c[-1] - w0) + (c[1] - w0));
#pragma unroll
        for (int m = 2; m <= R; ++m) lap = fmaf(a.cxm[m - 1], (c[-m] - w0) + (c[m] - w0), lap);
#pragma unroll
        for (int m = 1; m <= R; ++m)
            lap = fmaf(a.czm[m - 1], (w[R - m] - w0) + (w[R + m] - w0), lap);
        float vn = fmaf(ka[r], lap, ab[r] * vi[r]);
        float un = w0 + vn;
        const int z = zr + r;
        if (colok && z < a.NZ) {
            if (z == sz && x == sx) {
                // point source: + kappa A s at the source cell (increment and field)
                const float d = ka[r] * dev::ricker_scaled(a.j, a);
                vn += d;
                un += d;
            }
            const size_t i = (size_t)z * a.NXp + x;
            ub[i] = un;
            vb[i] = vn;
            if (STORE) rb[i] = lap;
        }
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) w[k] = w[k + 1];
    }
}

// ------------------------------------------------------------------ column quads
// The same steps with a thread owning four adjacent columns x .. x+3 (x a
// multiple of 4) and QR rows: 16-byte loads of the per-cell operands and
// 16-byte stores of the new level, the increment and the record, the
// stencil's centre row as one 16-byte shared-memory load and its x arms as
// 8- (4th order) or 16-byte (8th order) loads.  Per cell the operations and
// their order are those of k_tile_fwd / k_tile_adj, so the results are the
// same bits.  A quad that reaches the pad columns (x + 3 >= NX, < NXp) writes
// them too: their tables are zero, so u and its increment stay zero there,
// and no step reads their record or imaging sums.
constexpr int QR = 2;                                   // rows a quad thread owns
constexpr int kQuadThreads = (TX / 4) * (TZ / QR);      // 256

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float &q4(float4 &v, int q) { return (&v.x)[q]; }
__device__ __forceinline__ float q4c(const float4 &v, int q) { return (&v.x)[q]; }

// the row of u around the quad: u[x - R .. x + 3 + R] (centre at e[R .. R + 3])
template <int R>
__device__ __forceinline__ void row_arms(const float *c, float (&e)[4 + 2 * R])
{
    const float4 m = ld4(c);
    if (R == 2) {
        const float2 l = *reinterpret_cast<const float2 *>(c - 2);
        const float2 r = *reinterpret_cast<const float2 *>(c + 4);
        e[0] = l.x; e[1] = l.y; e[6] = r.x; e[7] = r.y;
    } else {
        const float4 l = ld4(c - 4), r = ld4(c + 4);
        e[0] = l.x; e[1] = l.y; e[2] = l.z; e[3] = l.w;
        e[8] = r.x; e[9] = r.y; e[10] = r.z; e[11] = r.w;
    }
    e[R] = m.x; e[R + 1] = m.y; e[R + 2] = m.z; e[R + 3] = m.w;
}

template <int R, int TOPBC, bool STORE>
__global__ void __launch_bounds__(kQuadThreads) k_tile_fwd4(const __grid_constant__ CUtensorMap tm,
                                                            const __grid_constant__ TileArgs a)
{
    constexpr int HZ = halo_rows<R>();
    __shared__ __align__(128) float tile[HZ * HX];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x, tq = tid % (TX / 4), g = tid / (TX / 4);
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, bs = blockIdx.z;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    if (tid == 0) mbar_init(&mbar);
    __syncthreads();
    if (tid == 0 && !a.withhold) tile_load(tile, &mbar, &tm, x0 - 4, z0 - R, bs, HZ * HX * sizeof(float));

    const int x = x0 + 4 * tq, zr = z0 + g * QR;
    const bool quadok = x < a.NXp;
    const size_t plane = (size_t)a.NZ * a.NXp;
    const float *kab = a.ka + (size_t)b * plane, *abb = a.ab + (size_t)b * plane;
    float *vb = a.vinc + (size_t)bs * plane;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ka[QR], ab[QR], vi[QR];
#pragma unroll
    for (int r = 0; r < QR; ++r) {
        const int z = zr + r;
        const bool ok = quadok && z < a.NZ;
        const size_t i = (size_t)z * a.NXp + x;
        ka[r] = ok ? ld4(kab + i) : zero4;
        ab[r] = ok ? ld4(abb + i) : zero4;
        vi[r] = ok ? ld4(vb + i) : zero4;
    }
    if (!tile_wait(&mbar, a.status, a.wait_polls)) return;
    if (TOPBC == 1 && z0 == 0) {
        for (int c = tid; c < HX; c += kQuadThreads) {
#pragma unroll
            for (int k = 1; k <= R; ++k) tile[(R - k) * HX + c] = tile[(R + k) * HX + c];
        }
        __syncthreads();
    }
    if (a.d_syn && a.j > 0 && z0 <= a.rzmax && z0 + TZ > a.rzmin) {
        for (int r = tid; r < a.nr; r += kQuadThreads) {
            const int pz = a.rec[r] >> 16, px = a.rec[r] & 0xffff;
            if (pz >= z0 && pz < z0 + TZ && px >= x0 && px < x0 + TX)
                a.d_syn[((size_t)bs * a.nr + r) * a.nt + a.j - 1] =
                    tile[(pz - z0 + R) * HX + px - x0 + 4];
        }
    }
    if (a.ckpt && a.j % a.ckpt_every == 0) {
        const size_t cells = (size_t)a.NZ * a.NX;
        float *st = a.ckpt + ((size_t)(a.j / a.ckpt_every) * gridDim.z + bs) * 2 * cells;
        // a quad wholly inside the grid goes out as two 16-byte stores when
        // the rows of the slot start on 16-byte boundaries (NX a multiple of
        // 4); otherwise cell by cell
        const bool whole = (a.NX & 3) == 0 && x + 3 < a.NX;
#pragma unroll
        for (int r = 0; r < QR; ++r) {
            const int z = zr + r;
            if (z >= a.NZ) continue;
            const float *t = tile + (z - z0 + R) * HX + 4 * tq + 4;
            if (whole) {
                st4(st + (size_t)z * a.NX + x, ld4(t));
                st4(st + cells + (size_t)z * a.NX + x, vi[r]);
                continue;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (x + q < a.NX) {
                    st[(size_t)z * a.NX + x + q] = t[q];
                    st[cells + (size_t)z * a.NX + x + q] = q4c(vi[r], q);
                }
            }
        }
    }

    const int sp = a.src[s], sz = sp >> 16, sx = sp & 0xffff;
    float *ub = a.unext + (size_t)bs * plane;
    float *rb = STORE ? a.rec_out + ((size_t)bs * a.rec_planes + (a.j - a.rec_base)) * plane
                      : nullptr;
    const float *cp = tile + (g * QR + R) * HX + 4 * tq + 4;
    float4 w[2 * R + 1];     // z window: w[R + k] = row z + k, four columns
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) w[k] = ld4(cp + (k - R) * HX);
#pragma unroll
    for (int r = 0; r < QR; ++r) {
        const float *c = cp + r * HX;
        w[2 * R] = ld4(c + R * HX);
        float e[4 + 2 * R];
        row_arms<R>(c, e);
        float4 lap4, vn4, un4;
        const int z = zr + r;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float w0 = e[R + q];
            float lap = a.cxm[0] * ((e[R + q - 1] - w0) + (e[R + q + 1] - w0));
#pragma unroll
            for (int m = 2; m <= R; ++m)
                lap = fmaf(a.cxm[m - 1], (e[R + q - m] - w0) + (e[R + q + m] - w0), lap);
#pragma unroll
            for (int m = 1; m <= R; ++m)
                lap = fmaf(a.czm[m - 1], (q4c(w[R - m], q) - w0) + (q4c(w[R + m], q) - w0), lap);
            float vn = fmaf(q4c(ka[r], q), lap, q4c(ab[r], q) * q4c(vi[r], q));
            float un = w0 + vn;
            if (z == sz && x + q == sx) {
                // point source: + kappa A s at the source cell (increment and field)
                const float d = q4c(ka[r], q) * dev::ricker_scaled(a.j, a);
                vn += d;
                un += d;
            }
            q4(lap4, q) = lap;
            q4(vn4, q) = vn;
            q4(un4, q) = un;
        }
        if (quadok && z < a.NZ) {
            const size_t i = (size_t)z * a.NXp + x;
            st4(ub + i, un4);
            st4(vb + i, vn4);
            if (STORE) st4(rb + i, lap4);
        }
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) w[k] = w[k + 1];
    }
}

template <int R, int TOPBC>
__global__ void __launch_bounds__(kQuadThreads) k_tile_adj4(const __grid_constant__ CUtensorMap tm,
                                                            const __grid_constant__ TileArgs a)
{
    constexpr int HZ = halo_rows<R>();
    __shared__ __align__(128) float tile[HZ * HX];
    __shared__ __align__(16) float inj[TZ * TX];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x, tq = tid % (TX / 4), g = tid / (TX / 4);
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, bs = blockIdx.z;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    if (tid == 0) mbar_init(&mbar);
    __syncthreads();
    if (tid == 0 && !a.withhold) tile_load(tile, &mbar, &tm, x0 - 4, z0 - R, bs, HZ * HX * sizeof(float));

    const int x = x0 + 4 * tq, zr = z0 + g * QR;
    const bool quadok = x < a.NXp;
    const size_t plane = (size_t)a.NZ * a.NXp;
    const float *kab = a.ka + (size_t)b * plane, *abb = a.ab + (size_t)b * plane;
    float *wb = a.vinc + (size_t)bs * plane, *accb = a.acc + (size_t)bs * plane;
    float *pn = a.unext + (size_t)bs * plane;
    const float *rb =
        a.rec_in + ((size_t)bs * a.rec_planes + (a.nt - 1 - a.j - a.rec_base)) * plane;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ka[QR], ab[QR], wi[QR], ac[QR], sv[QR];
#pragma unroll
    for (int r = 0; r < QR; ++r) {
        const int z = zr + r;
        const bool ok = quadok && z < a.NZ;
        const size_t i = (size_t)z * a.NXp + x;
        ka[r] = ok ? ld4(kab + i) : zero4;
        ab[r] = ok ? ld4(abb + i) : zero4;
        wi[r] = ok ? ld4(wb + i) : zero4;
        ac[r] = ok ? ld4(accb + i) : zero4;
        sv[r] = ok ? ld4(rb + i) : zero4;
    }
    const bool has_rec = z0 <= a.rzmax && z0 + TZ > a.rzmin;
    if (has_rec) {
#pragma unroll
        for (int r = 0; r < QR; ++r) st4(inj + (g * QR + r) * TX + 4 * tq, zero4);
    }
    if (!tile_wait(&mbar, a.status, a.wait_polls)) return;
    if (has_rec) {
        for (int r = tid; r < a.nr; r += kQuadThreads) {
            const int pz = a.rec[r] >> 16, px = a.rec[r] & 0xffff;
            if (pz >= z0 && pz < z0 + TZ && px >= x0 && px < x0 + TX)
                inj[(pz - z0) * TX + px - x0] =
                    a.adj[((size_t)bs * a.nr + r) * a.nt + (a.nt - 1 - a.j)];
        }
        __syncthreads();
    }

    const int sp = a.src[s], sz = sp >> 16, sx = sp & 0xffff;
    const float *cp = tile + (g * QR + R) * HX + 4 * tq + 4;
    float4 w[2 * R + 1];
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) w[k] = ld4(cp + (k - R) * HX);
#pragma unroll
    for (int r = 0; r < QR; ++r) {
        const float *c = cp + r * HX;
        w[2 * R] = ld4(c + R * HX);
        float e[4 + 2 * R];
        row_arms<R>(c, e);
        const int z = zr + r;
        const float4 in4 = has_rec ? ld4(inj + (g * QR + r) * TX + 4 * tq) : zero4;
        float4 pn4, wn4, ac4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float w0 = e[R + q];
            float lap = a.cxm[0] * ((e[R + q - 1] - w0) + (e[R + q + 1] - w0));
#pragma unroll
            for (int m = 2; m <= R; ++m)
                lap = fmaf(a.cxm[m - 1], (e[R + q - m] - w0) + (e[R + q + m] - w0), lap);
#pragma unroll
            for (int m = 1; m <= R; ++m)
                lap = fmaf(a.czm[m - 1], (q4c(w[R - m], q) - w0) + (q4c(w[R + m], q) - w0), lap);
            if (TOPBC == 1 && z0 == 0) {
                // transpose of the mirrored top: rows 0..R-z reflect onto row z
                // (grid rows 1..R may lie in this thread's rows or the next ones')
#pragma unroll
                for (int zz = 1; zz <= R; ++zz) {
                    if (z == zz) {
                        float extra = 0.f;
#pragma unroll
                        for (int r0 = 0; r0 <= R - zz; ++r0)
                            extra = fmaf(a.czm[r0 + zz - 1], q4c(w[R + r0 - zz], q), extra);
                        lap += extra;
                    }
                }
            }
            float wn = fmaf(q4c(ka[r], q), lap, q4c(ab[r], q) * q4c(wi[r], q));
            if (has_rec) wn = fmaf(q4c(ka[r], q), q4c(in4, q), wn);
            const float pnv = w0 + wn;
            q4(pn4, q) = pnv;
            q4(wn4, q) = wn;
            q4(ac4, q) = fmaf(pnv, q4c(sv[r], q), q4c(ac[r], q));
            if (quadok && z < a.NZ && z == sz && x + q == sx)
                a.acc_src[bs] = fmaf(pnv, dev::ricker_scaled(a.nt - 1 - a.j, a), a.acc_src[bs]);
        }
        if (quadok && z < a.NZ) {
            const size_t i = (size_t)z * a.NXp + x;
            st4(pn + i, pn4);
            st4(wb + i, wn4);
            st4(accb + i, ac4);
        }
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) w[k] = w[k + 1];
    }
}

// d[:, nt-1] = u^nt at the receivers
__global__ void k_tile_gather(const float *__restrict__ u, const int *__restrict__ rec, int nbs,
                              int nr, int nt, size_t plane, int NXp, float *__restrict__ d_syn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbs * nr) return;
    const int bs = i / nr, r = i - (i / nr) * nr;
    const int pz = rec[r] >> 16, px = rec[r] & 0xffff;
    d_syn[((size_t)bs * nr + r) * nt + nt - 1] = u[(size_t)bs * plane + (size_t)pz * NXp + px];
}

// state at a checkpoint slot ([bs][2][NZ][NX]) into the field and increment
__global__ void k_tile_resume(const float *__restrict__ st, int nbs, int NZ, int NX, int NXp,
                              float *__restrict__ u, float *__restrict__ v)
{
    const size_t cells = (size_t)NZ * NX, n = (size_t)nbs * cells;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t bs = i / cells, c = i - bs * cells;
        const int z = (int)(c / NX), x = (int)(c - (c / NX) * NX);
        const size_t o = bs * (size_t)NZ * NXp + (size_t)z * NXp + x;
        u[o] = st[bs * 2 * cells + c];
        v[o] = st[bs * 2 * cells + cells + c];
    }
}

// ------------------------------------------------------------------ adjoint step
// Increment form of the adjoint recurrence (the forward's form with L^T):
//   w^{j+1/2} = A B w^{j-1/2} + kappa A (L^T psi^j + q^j),  psi^{j+1} = psi^j + w^{j+1/2},
// q^j the adjoint source r^{nt-1-j} at the receivers.  Over thousands of
// steps the standard form 2A psi^j - A B psi^{j-1} loses the slowly varying
// part of psi to float32 round-off, as the forward's standard form does.
// With the mirrored top, L^T adds the reflected weights back onto rows
// 1..R: (L^T psi)_k += sum_{r=0}^{R-k} c_{r+k} psi_r.
template <int R, int TOPBC, int TRW>
__global__ void __launch_bounds__(tile_threads<TRW>()) k_tile_adj(const __grid_constant__ CUtensorMap tm,
                                                       const __grid_constant__ TileArgs a)
{
    constexpr int HZ = halo_rows<R>();
    __shared__ __align__(128) float tile[HZ * HX];
    __shared__ float inj[TZ * TX];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x, tx = tid % TX, g = tid / TX;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, bs = blockIdx.z;
    const int b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    if (tid == 0) mbar_init(&mbar);
    __syncthreads();
    if (tid == 0 && !a.withhold) tile_load(tile, &mbar, &tm, x0 - 4, z0 - R, bs, HZ * HX * sizeof(float));

    const int x = x0 + tx, zr = z0 + g * TRW;
    const bool colok = x < a.NX;
    const size_t plane = (size_t)a.NZ * a.NXp;
    const float *kab = a.ka + (size_t)b * plane, *abb = a.ab + (size_t)b * plane;
    float *wb = a.vinc + (size_t)bs * plane, *accb = a.acc + (size_t)bs * plane;
    float *pn = a.unext + (size_t)bs * plane;
    const float *rb =
        a.rec_in + ((size_t)bs * a.rec_planes + (a.nt - 1 - a.j - a.rec_base)) * plane;
    float ka[TRW], ab[TRW], wi[TRW], ac[TRW], sv[TRW];
#pragma unroll
    for (int r = 0; r < TRW; ++r) {
        const int z = zr + r;
        const bool ok = colok && z < a.NZ;
        const size_t i = (size_t)z * a.NXp + x;
        ka[r] = ok ? kab[i] : 0.f;
        ab[r] = ok ? abb[i] : 0.f;
        wi[r] = ok ? wb[i] : 0.f;
        ac[r] = ok ? accb[i] : 0.f;
        sv[r] = ok ? rb[i] : 0.f;
    }
    // adjoint source of the receivers inside this tile
    const bool has_rec = z0 <= a.rzmax && z0 + TZ > a.rzmin;
    if (has_rec) {
#pragma unroll
        for (int r = 0; r < TRW; ++r) inj[(g * TRW + r) * TX + tx] = 0.f;
    }
    if (!tile_wait(&mbar, a.status, a.wait_polls)) return;
    if (has_rec) {
        for (int r = tid; r < a.nr; r += tile_threads<TRW>()) {
            const int pz = a.rec[r] >> 16, px = a.rec[r] & 0xffff;
            if (pz >= z0 && pz < z0 + TZ && px >= x0 && px < x0 + TX)
                inj[(pz - z0) * TX + px - x0] =
                    a.adj[((size_t)bs * a.nr + r) * a.nt + (a.nt - 1 - a.j)];
        }
        __syncthreads();
    }

    const int sp = a.src[s], sz = sp >> 16, sx = sp & 0xffff;
    const float *cp = tile + (g * TRW + R) * HX + tx + 4;
    float w[2 * R + 1];     // z window: w[R + k] = row z + k
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) w[k] = cp[(k - R) * HX];
#pragma unroll
    for (int r = 0; r < TRW; ++r) {
        const float *c = cp + r * HX;
        w[2 * R] = c[R * HX];
        const float w0 = w[R];
        const int z = zr + r;
        float lap = a.cxm[0] * ((c[-1] - w0) + (c[1] - w0));
#pragma unroll
        for (int m = 2; m <= R; ++m) lap = fmaf(a.cxm[m - 1], (c[-m] - w0) + (c[m] - w0), lap);
#pragma unroll
        for (int m = 1; m <= R; ++m)
            lap = fmaf(a.czm[m - 1], (w[R - m] - w0) + (w[R + m] - w0), lap);
        if (TOPBC == 1 && r >= 1 && r <= R && zr == 0) {
            // transpose of the mirrored top: rows 0..R-r reflect onto row r
            // (rows 1..R of the grid are rows 1..R of the first row group)
            float extra = 0.f;
#pragma unroll
            for (int r0 = 0; r0 <= R - r; ++r0) extra = fmaf(a.czm[r0 + r - 1], w[R + r0 - r], extra);
            lap += extra;
        }
        float wn = fmaf(ka[r], lap, ab[r] * wi[r]);
        if (has_rec) wn = fmaf(ka[r], inj[(g * TRW + r) * TX + tx], wn);
        const float pnv = w0 + wn;
        if (colok && z < a.NZ) {
            const size_t i = (size_t)z * a.NXp + x;
            pn[i] = pnv;
            wb[i] = wn;
            accb[i] = fmaf(pnv, sv[r], ac[r]);
            if (z == sz && x == sx)
                a.acc_src[bs] = fmaf(pnv, dev::ricker_scaled(a.nt - 1 - a.j, a), a.acc_src[bs]);
        }
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) w[k] = w[k + 1];
    }
}

// dJ/dv_pad = 2 acc / v_pad, folded onto the physical cells (transpose of the
// edge replication: each physical cell sums the padded cells that copy it,
// columns then rows in increasing order), per (model, shot)
__global__ void k_tile_fold(const __grid_constant__ PropArgs a, int NXp,
                            const float *__restrict__ acc, const float *__restrict__ acc_src,
                            float *__restrict__ gshot)
{
    const int bs = blockIdx.y, b = bs / a.ns, s = bs - (bs / a.ns) * a.ns;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nz * a.nx) return;
    const int iz = i / a.nx, ix = i - (i / a.nx) * a.nx;
    const float v = a.v[(size_t)b * a.nz * a.nx + i];
    const int r0 = iz, r1 = (iz == a.nz - 1) ? a.NZ - 1 : iz;
    const int c0 = (ix == 0) ? 0 : ix + a.nb, c1 = (ix == a.nx - 1) ? a.NX - 1 : ix + a.nb;
    const int sz = a.src_pz[s], sx = a.src_px[s];
    const float *ab = acc + (size_t)bs * a.NZ * NXp;
    float sum = 0.f;
    for (int pz = r0; pz <= r1; ++pz) {
        float row = 0.f;
        for (int px = c0; px <= c1; ++px) {
            float gpad = 2.f * ab[(size_t)pz * NXp + px] / v;
            if (pz == sz && px == sx) gpad += 2.f * acc_src[bs] / v;
            row += gpad;
        }
        sum += row;
    }
    gshot[(size_t)bs * a.nz * a.nx + i] = sum;
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3D map [nbs][NZ][NXp] of float32 with the halo-tile box of radius R
bool make_map(CUtensorMap *m, float *base, int nbs, int NZ, int NXp, int R)
{
    auto enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)NXp, (cuuint64_t)NZ, (cuuint64_t)nbs};
    const cuuint64_t strides[2] = {(cuuint64_t)NXp * 4, (cuuint64_t)NZ * NXp * 4};
    const cuuint32_t box[3] = {HX, (cuuint32_t)(TZ + 2 * R), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TileBufs {
    float *u[2], *v, *p[2], *w, *acc, *ka, *ab, *acc_src;
    int *rec, *src;
};

TileBufs tile_bufs(const Plan &pl, unsigned char *ws)
{
    TileBufs t;
    t.u[0] = (float *)(ws + pl.ws_t_u0);
    t.u[1] = (float *)(ws + pl.ws_t_u1);
    t.v = (float *)(ws + pl.ws_t_v);
    t.p[0] = (float *)(ws + pl.ws_t_p0);
    t.p[1] = (float *)(ws + pl.ws_t_p1);
    t.w = (float *)(ws + pl.ws_t_w);
    t.acc = (float *)(ws + pl.ws_t_acc);
    t.ka = (float *)(ws + pl.ws_t_ka);
    t.ab = (float *)(ws + pl.ws_t_ab);
    t.acc_src = (float *)(ws + pl.ws_t_accsrc);
    t.rec = (int *)(ws + pl.ws_t_rec);
    t.src = (int *)(ws + pl.ws_t_src);
    return t;
}

TileArgs tile_args(const Plan &pl, const PropArgs &a, const TileBufs &t)
{
    TileArgs s{};
    s.wait_polls = kWaitLimit;
    s.nz = a.nz; s.nx = a.nx; s.nb = a.nb; s.NZ = a.NZ; s.NX = a.NX; s.NXp = pl.NXp;
    s.nt = a.nt; s.ns = a.ns; s.nr = a.nr;
    s.dtd = a.dtd; s.t0d = a.t0d; s.ex0d = a.ex0d; s.ez0d = a.ez0d;
    s.c0 = a.c0; s.cx1 = a.cx1; s.cx2 = a.cx2; s.cz1 = a.cz1; s.cz2 = a.cz2;
    s.ex0 = a.ex0; s.ez0 = a.ez0; s.inv_nb = a.inv_nb; s.fp = a.fp; s.src_scale = a.src_scale;
    // second-difference weights of offsets 1..R (4th order: 4/3, -1/12; 8th
    // order: 8/5, -1/5, 8/315, -1/560), divided by h^2
    static const double w4[4] = {4.0 / 3.0, -1.0 / 12.0, 0.0, 0.0};
    static const double w8[4] = {8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    const double *wm = pl.p.space_order == 8 ? w8 : w4;
    const double ix2 = 1.0 / ((double)pl.p.dx * pl.p.dx), iz2 = 1.0 / ((double)pl.p.dz * pl.p.dz);
    for (int m = 0; m < 4; ++m) {
        s.cxm[m] = (float)(wm[m] * ix2);
        s.czm[m] = (float)(wm[m] * iz2);
    }
    int zmin = 1 << 30, zmax = -1;
    for (int i = 0; i < a.nr; ++i) {
        zmin = a.rec_pz[i] < zmin ? a.rec_pz[i] : zmin;
        zmax = a.rec_pz[i] > zmax ? a.rec_pz[i] : zmax;
    }
    s.rzmin = zmin;
    s.rzmax = zmax;
    s.ka = t.ka; s.ab = t.ab; s.rec = t.rec; s.src = t.src;
    s.status = a.status;
    return s;
}

cudaError_t setup(const Plan &pl, const PropArgs &a, const TileBufs &t, cudaStream_t st)
{
    const size_t plane = (size_t)pl.NZ * pl.NXp;
    dim3 grid((unsigned)((plane + 255) / 256 < 1024 ? (plane + 255) / 256 : 1024), pl.p.batch);
    k_tile_setup<<<grid, 256, 0, st>>>(a, pl.NXp, t.ka, t.ab, t.rec, t.src);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_fold(const Plan &pl, const PropArgs &a, unsigned char *ws, cudaStream_t st)
{
    const int nbs = pl.p.batch * pl.p.ns;
    const TileBufs t = tile_bufs(pl, ws);
    const dim3 fg((pl.p.nz * pl.p.nx + 255) / 256, nbs);
    k_tile_fold<<<fg, 256, 0, st>>>(a, pl.NXp, t.acc, t.acc_src, a.gshot);
    return cudaGetLastError();
}

cudaError_t launch_tiled(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                         cudaStream_t st, bool wait_check)
{
    const int nbs = pl.p.batch * pl.p.ns;
    const size_t plane = (size_t)pl.NZ * pl.NXp, field = (size_t)nbs * plane * sizeof(float);
    const TileBufs t = tile_bufs(pl, ws);
    cudaError_t e = setup(pl, a, t, st);
    if (e != cudaSuccess) return e;
    TileArgs s = tile_args(pl, a, t);
    if (wait_check) {   // the self-check: no tile is loaded, every wait runs out quickly
        s.withhold = 1;
        s.wait_polls = 1024;
    }
    s.rec_base = a.rec_base;
    s.rec_planes = a.rec_planes;
    const dim3 grid((pl.NX + TX - 1) / TX, (pl.NZ + TZ - 1) / TZ, nbs);
    const int tb = pl.p.top_bc;
    const int R = pl.p.space_order == 8 ? 4 : 2;
    CUtensorMap maps[2];
    if (!adj) {
        const int jb = a.j_begin;
        if (a.resume) {
            e = cudaMemsetAsync(t.u[jb & 1], 0, field, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(t.v, 0, field, st);
            if (e != cudaSuccess) return e;
            k_tile_resume<<<1024, 256, 0, st>>>(a.resume + 0, nbs, pl.NZ, pl.NX, pl.NXp,
                                                t.u[jb & 1], t.v);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        } else {
            e = cudaMemsetAsync(t.u[jb & 1], 0, field, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(t.v, 0, field, st);
            if (e != cudaSuccess) return e;
        }
        // the other level's pad columns and dead cells must read as zero too
        e = cudaMemsetAsync(t.u[(jb + 1) & 1], 0, field, st);
        if (e != cudaSuccess) return e;
        if (!make_map(&maps[0], t.u[0], nbs, pl.NZ, pl.NXp, R) ||
            !make_map(&maps[1], t.u[1], nbs, pl.NZ, pl.NXp, R))
            return cudaErrorNotSupported;
        s.vinc = t.v;
        s.rec_out = a.snap;
        s.d_syn = a.d_syn;
        s.ckpt = a.ckpt;
        s.ckpt_every = a.ckpt_every;
        const bool store = a.snap != nullptr;
        for (int j = jb; j < a.j_end; ++j) {
            s.j = j;
            s.unext = t.u[(j + 1) & 1];
#define FWI_TFWD(RR, TB, ST, TR)                                                              \
    k_tile_fwd<RR, TB, ST, TR><<<grid, tile_threads<TR>(), 0, st>>>(maps[j & 1], s)
#define FWI_TFWD_R(TR)                                                                         \
    if (R == 4) {                                                                              \
        if (store) tb ? FWI_TFWD(4, 1, true, TR) : FWI_TFWD(4, 0, true, TR);                   \
        else tb ? FWI_TFWD(4, 1, false, TR) : FWI_TFWD(4, 0, false, TR);                       \
    } else {                                                                                   \
        if (store) tb ? FWI_TFWD(2, 1, true, TR) : FWI_TFWD(2, 0, true, TR);                   \
        else tb ? FWI_TFWD(2, 1, false, TR) : FWI_TFWD(2, 0, false, TR);                       \
    }
            if (pl.tile_quads) {
#define FWI_TFWD4(RR, TB, ST) k_tile_fwd4<RR, TB, ST><<<grid, kQuadThreads, 0, st>>>(maps[j & 1], s)
                if (R == 4) {
                    if (store) tb ? FWI_TFWD4(4, 1, true) : FWI_TFWD4(4, 0, true);
                    else tb ? FWI_TFWD4(4, 1, false) : FWI_TFWD4(4, 0, false);
                } else {
                    if (store) tb ? FWI_TFWD4(2, 1, true) : FWI_TFWD4(2, 0, true);
                    else tb ? FWI_TFWD4(2, 1, false) : FWI_TFWD4(2, 0, false);
                }
#undef FWI_TFWD4
            } else if (pl.tile_rows == 4) {
                FWI_TFWD_R(4)
            } else {
                FWI_TFWD_R(8)
            }
#undef FWI_TFWD_R
#undef FWI_TFWD
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (a.d_syn && a.j_end == a.nt) {
            const int n = nbs * pl.p.nr;
            k_tile_gather<<<(n + 255) / 256, 256, 0, st>>>(t.u[a.nt & 1], t.rec, nbs, pl.p.nr,
                                                          a.nt, plane, pl.NXp, a.d_syn);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // adjoint window [j_begin, j_end); the levels and sums persist in the
    // workspace between windows
    const int jb = a.j_begin;
    if (jb == 0) {
        e = cudaMemsetAsync(t.p[0], 0, field, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.p[1], 0, field, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.w, 0, field, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.acc, 0, field, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.acc_src, 0, (size_t)nbs * sizeof(float), st);
        if (e != cudaSuccess) return e;
    }
    if (!make_map(&maps[0], t.p[0], nbs, pl.NZ, pl.NXp, R) ||
        !make_map(&maps[1], t.p[1], nbs, pl.NZ, pl.NXp, R))
        return cudaErrorNotSupported;
    s.acc = t.acc;
    s.acc_src = t.acc_src;
    s.adj = a.adj;
    s.rec_in = a.snap;
    s.vinc = t.w;
    for (int j = jb; j < a.j_end; ++j) {
        s.j = j;
        s.unext = t.p[(j + 1) & 1];
#define FWI_TADJ(RR, TB, TR) k_tile_adj<RR, TB, TR><<<grid, tile_threads<TR>(), 0, st>>>(maps[j & 1], s)
#define FWI_TADJ4(RR, TB) k_tile_adj4<RR, TB><<<grid, kQuadThreads, 0, st>>>(maps[j & 1], s)
        if (pl.tile_quads) {
            if (R == 4) tb ? FWI_TADJ4(4, 1) : FWI_TADJ4(4, 0);
            else tb ? FWI_TADJ4(2, 1) : FWI_TADJ4(2, 0);
        } else if (pl.tile_rows == 4) {
            if (R == 4) tb ? FWI_TADJ(4, 1, 4) : FWI_TADJ(4, 0, 4);
            else tb ? FWI_TADJ(2, 1, 4) : FWI_TADJ(2, 0, 4);
        } else {
            if (R == 4) tb ? FWI_TADJ(4, 1, 8) : FWI_TADJ(4, 0, 8);
            else tb ? FWI_TADJ(2, 1, 8) : FWI_TADJ(2, 0, 8);
        }
#undef FWI_TADJ4
#undef FWI_TADJ
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.j_end == a.nt) {
        const dim3 fg((pl.p.nz * pl.p.nx + 255) / 256, nbs);
        k_tile_fold<<<fg, 256, 0, st>>>(a, pl.NXp, t.acc, t.acc_src, a.gshot);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fwi
