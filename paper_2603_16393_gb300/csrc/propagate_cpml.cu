// propagate_cpml.cu -- forward and adjoint solves with a convolutional PML as
// the absorbing layer (fwi_problem.absorber = FWI_ABSORBER_CPML): the layer
// stretches d/dx and d/dz, s = 1 + sigma/(i omega), and each 1/s convolution
// is a memory variable advanced once per step (4th-order stencils, zero
// values outside the padded grid):
//
//   psi_x  = b_x psi_x  + a_x Dx u^j
//   h_x    = Dxx u^j + Dx psi_x
//   zeta_x = b_x zeta_x + a_x h_x                       (same in z)
//   B^j    = h_x + zeta_x + h_z + zeta_z + s^j
//   w      = w + kappa B^j,  u^{j+1} = u^j + w           (increment form)
//
// b = exp(-sigma dt), a = b - 1, sigma = d0 (d/nb)^2 in the d-th cell into
// the layer, d0 = 3 v_ref ln(1/R) / (2 nb h); both formed in double.  The
// adjoint is the exact transpose step by step (Dx^T = -Dx, Dxx^T = Dxx with
// zero outside values):
//
//   Bb = kappa mu^{j+1};  acc += Bb B^j           (dJ/dv_pad = 2 acc / v_pad)
//   zt = zb_x + Bb,  hb_x = Bb + a_x zt,  zb_x = b_x zt
//   pt = pb_x - Dx hb_x,  t_x = a_x pt,   pb_x = b_x pt
//   G  = Dxx hb_x + Dzz hb_z - Dx t_x - Dz t_z + R^T r^{j-1}
//   nu = nu + G,  mu^j = mu^{j+1} + nu                (nu = mu^j - mu^{j+1})
//
// Global-memory fields, 32 x 8 threads per block over one (model, shot) grid
// (blockIdx.z); two launches per forward step, three per adjoint step.  A
// variant of the physics, not a bandwidth-tuned path.
#include <cuda_runtime.h>

#include <cmath>

#include "fwi_device.cuh"
#include "fwi_internal.cuh"

namespace fwi {

namespace {

using dev::ricker_scaled;

constexpr int BX = 32, BZ = 8;

struct CpmlArgs {
    float d1x, d2x, d1z, d2z;             // first-difference weights 8/(12h), 1/(12h)
    size_t field;                         // floats per (model, shot) grid
    float *u0, *u1, *w;                   // forward: two levels, increment
    float *p_x, *p_z, *z_x, *z_z;         // memory variables (adjoint: their adjoints)
    float *hb_x, *hb_z, *t_x, *t_z, *acc; // adjoint only
    float *kap;                           // [B][NZ][NX]
    float *ax, *bx, *az, *bz;             // [NX], [NX], [NZ], [NZ]
    int *rmap;                            // [NZ][NX]: receiver index or -1
};

// value of f at (z, x) of one grid, 0 outside
__device__ __forceinline__ float at(const float *f, int z, int x, int NZ, int NX)
{
    return (z >= 0 && z < NZ && x >= 0 && x < NX) ? f[z * NX + x] : 0.f;
}

__device__ __forceinline__ float dfx(const float *f, int z, int x, int NZ, int NX, float d1,
                                     float d2)
{
    return d1 * (at(f, z, x + 1, NZ, NX) - at(f, z, x - 1, NZ, NX)) -
           d2 * (at(f, z, x + 2, NZ, NX) - at(f, z, x - 2, NZ, NX));
}

__device__ __forceinline__ float dfz(const float *f, int z, int x, int NZ, int NX, float d1,
                                     float d2)
{
    return d1 * (at(f, z + 1, x, NZ, NX) - at(f, z - 1, x, NZ, NX)) -
           d2 * (at(f, z + 2, x, NZ, NX) - at(f, z - 2, x, NZ, NX));
}

// second differences on neighbour differences (f0 = f(z, x))
__device__ __forceinline__ float d2x(const float *f, float f0, int z, int x, int NZ, int NX,
                                     float c1, float c2)
{
    return c1 * ((at(f, z, x - 1, NZ, NX) - f0) + (at(f, z, x + 1, NZ, NX) - f0)) +
           c2 * ((at(f, z, x - 2, NZ, NX) - f0) + (at(f, z, x + 2, NZ, NX) - f0));
}

__device__ __forceinline__ float d2z(const float *f, float f0, int z, int x, int NZ, int NX,
                                     float c1, float c2)
{
    return c1 * ((at(f, z - 1, x, NZ, NX) - f0) + (at(f, z + 1, x, NZ, NX) - f0)) +
           c2 * ((at(f, z - 2, x, NZ, NX) - f0) + (at(f, z + 2, x, NZ, NX) - f0));
}

// kappa = (v_pad dt)^2 per model and cell; profiles; receiver map (-1)
__global__ void k_cpml_setup(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c,
                             double d0x, double d0z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (i >= NZ * NX) return;
    const int pz = i / NX, px = i - (i / NX) * NX;
    const float vv = a.v[(size_t)b * a.nz * a.nx + min(pz, a.nz - 1) * a.nx +
                         min(max(px - a.nb, 0), a.nx - 1)];
    if (!(vv > 0.f && vv <= a.vmax)) set_status(a.status, FWI_ERR_UNSTABLE_CFL);
    const double vdt = (double)vv * a.dtd;
    c.kap[(size_t)b * NZ * NX + i] = (float)(vdt * vdt);
    if (b != 0) return;
    c.rmap[i] = -1;
    if (pz == 0) {   // column profile
        double cx = 0.0;
        if (px < a.nb) cx = (double)(a.nb - px);
        if (px > a.nb + a.nx - 1) cx = (double)(px - (a.nb + a.nx - 1));
        const double r = a.nb > 0 ? cx / a.nb : 0.0;
        const double bb = exp(-d0x * r * r * a.dtd);
        c.bx[px] = (float)bb;
        c.ax[px] = (float)(bb - 1.0);
    }
    if (px == 0) {   // row profile (bottom layer)
        const double cz = pz > a.nz - 1 ? (double)(pz - (a.nz - 1)) : 0.0;
        const double r = a.nb > 0 ? cz / a.nb : 0.0;
        const double bb = exp(-d0z * r * r * a.dtd);
        c.bz[pz] = (float)bb;
        c.az[pz] = (float)(bb - 1.0);
    }
}

__global__ void k_cpml_recmap(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.nr) c.rmap[a.rec_pz[i] * a.NX + a.rec_px[i]] = i;
}

// ---------------------------------------------------------------- forward
__global__ void __launch_bounds__(BX * BZ)
k_cpml_psi(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c, int j)
{
    const int x = blockIdx.x * BX + threadIdx.x, z = blockIdx.y * BZ + threadIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (x >= NX || z >= NZ) return;
    const float ax = c.ax[x], az = c.az[z];
    if (ax == 0.f && az == 0.f) return;
    const size_t o = (size_t)blockIdx.z * c.field;
    const float *u = ((j & 1) ? c.u1 : c.u0) + o;
    const int i = z * NX + x;
    if (ax != 0.f) c.p_x[o + i] = c.bx[x] * c.p_x[o + i] + ax * dfx(u, z, x, NZ, NX, c.d1x, c.d2x);
    if (az != 0.f) c.p_z[o + i] = c.bz[z] * c.p_z[o + i] + az * dfz(u, z, x, NZ, NX, c.d1z, c.d2z);
}

template <bool STORE>
__global__ void __launch_bounds__(BX * BZ)
k_cpml_step(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c, int j)
{
    const int x = blockIdx.x * BX + threadIdx.x, z = blockIdx.y * BZ + threadIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (x >= NX || z >= NZ) return;
    const int bs = blockIdx.z, b = bs / a.ns, s = bs - b * a.ns;
    const size_t o = (size_t)bs * c.field;
    const float *u = ((j & 1) ? c.u1 : c.u0) + o;
    float *un = ((j & 1) ? c.u0 : c.u1) + o;
    const int i = z * NX + x;
    const float u0 = u[i];
    const float hx = d2x(u, u0, z, x, NZ, NX, a.cx1, a.cx2) +
                     dfx(c.p_x + o, z, x, NZ, NX, c.d1x, c.d2x);
    const float hz = d2z(u, u0, z, x, NZ, NX, a.cz1, a.cz2) +
                     dfz(c.p_z + o, z, x, NZ, NX, c.d1z, c.d2z);
    const float zx = c.bx[x] * c.z_x[o + i] + c.ax[x] * hx;
    const float zz = c.bz[z] * c.z_z[o + i] + c.az[z] * hz;
    c.z_x[o + i] = zx;
    c.z_z[o + i] = zz;
    float B = (hx + zx) + (hz + zz);
    if (z == a.src_pz[s] && x == a.src_px[s]) B += ricker_scaled(j, a);
    const float w = c.w[o + i] + c.kap[(size_t)b * c.field + i] * B;
    c.w[o + i] = w;
    const float unew = u0 + w;
    un[i] = unew;
    if (STORE) a.snap[((size_t)bs * a.nt + j) * c.field + i] = B;
    const int r = c.rmap[i];
    if (r >= 0) a.d_syn[((size_t)bs * a.nr + r) * a.nt + j] = unew;
}

// ---------------------------------------------------------------- adjoint
__global__ void k_cpml_adj_init(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c)
{
    const int i = threadIdx.x + blockIdx.x * blockDim.x, bs = blockIdx.y;
    if (i >= a.nr) return;
    const float r = a.adj[((size_t)bs * a.nr + i) * a.nt + (a.nt - 1)];
    const size_t o = (size_t)bs * c.field + a.rec_pz[i] * a.NX + a.rec_px[i];
    c.u0[o] = r;   // mu^{nt}
    c.w[o] = r;    // nu = mu^{nt} - mu^{nt+1}
}

__global__ void __launch_bounds__(BX * BZ)
k_cpml_adj_a(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c, int j)
{
    const int x = blockIdx.x * BX + threadIdx.x, z = blockIdx.y * BZ + threadIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (x >= NX || z >= NZ) return;
    const int bs = blockIdx.z, b = bs / a.ns;
    const size_t o = (size_t)bs * c.field;
    const int i = z * NX + x;
    const float Bb = c.kap[(size_t)b * c.field + i] * c.u0[o + i];
    c.acc[o + i] += Bb * a.snap[((size_t)bs * a.nt + j) * c.field + i];
    const float ax = c.ax[x], az = c.az[z];
    float hx = Bb, hz = Bb;
    if (ax != 0.f) {
        const float zt = c.z_x[o + i] + Bb;
        hx = Bb + ax * zt;
        c.z_x[o + i] = c.bx[x] * zt;
    }
    if (az != 0.f) {
        const float zt = c.z_z[o + i] + Bb;
        hz = Bb + az * zt;
        c.z_z[o + i] = c.bz[z] * zt;
    }
    c.hb_x[o + i] = hx;
    c.hb_z[o + i] = hz;
}

__global__ void __launch_bounds__(BX * BZ)
k_cpml_adj_b(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c)
{
    const int x = blockIdx.x * BX + threadIdx.x, z = blockIdx.y * BZ + threadIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (x >= NX || z >= NZ) return;
    const size_t o = (size_t)blockIdx.z * c.field;
    const int i = z * NX + x;
    const float ax = c.ax[x], az = c.az[z];
    float tx = 0.f, tz = 0.f;
    if (ax != 0.f) {
        const float pt = c.p_x[o + i] - dfx(c.hb_x + o, z, x, NZ, NX, c.d1x, c.d2x);
        tx = ax * pt;
        c.p_x[o + i] = c.bx[x] * pt;
    }
    if (az != 0.f) {
        const float pt = c.p_z[o + i] - dfz(c.hb_z + o, z, x, NZ, NX, c.d1z, c.d2z);
        tz = az * pt;
        c.p_z[o + i] = c.bz[z] * pt;
    }
    c.t_x[o + i] = tx;
    c.t_z[o + i] = tz;
}

__global__ void __launch_bounds__(BX * BZ)
k_cpml_adj_c(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c, int j)
{
    const int x = blockIdx.x * BX + threadIdx.x, z = blockIdx.y * BZ + threadIdx.y;
    const int NZ = a.NZ, NX = a.NX;
    if (x >= NX || z >= NZ) return;
    const int bs = blockIdx.z;
    const size_t o = (size_t)bs * c.field;
    const int i = z * NX + x;
    const float *hx = c.hb_x + o, *hz = c.hb_z + o;
    float G = d2x(hx, hx[i], z, x, NZ, NX, a.cx1, a.cx2) + d2z(hz, hz[i], z, x, NZ, NX, a.cz1, a.cz2);
    G -= dfx(c.t_x + o, z, x, NZ, NX, c.d1x, c.d2x) + dfz(c.t_z + o, z, x, NZ, NX, c.d1z, c.d2z);
    const int r = c.rmap[i];
    if (r >= 0) G += a.adj[((size_t)bs * a.nr + r) * a.nt + (j - 1)];
    const float nu = c.w[o + i] + G;
    c.w[o + i] = nu;
    c.u0[o + i] += nu;
}

// dJ/dv = 2 acc / v_pad folded onto the physical grid (edge replication)
__global__ void k_cpml_fold(const __grid_constant__ PropArgs a, const __grid_constant__ CpmlArgs c)
{
    const int bs = blockIdx.y, b = bs / a.ns;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nz * a.nx) return;
    const int iz = i / a.nx, ix = i - (i / a.nx) * a.nx;
    const float v = a.v[(size_t)b * a.nz * a.nx + i];
    const int r1 = (iz == a.nz - 1) ? a.NZ - 1 : iz;
    const int c0 = (ix == 0) ? 0 : ix + a.nb, c1 = (ix == a.nx - 1) ? a.NX - 1 : ix + a.nb;
    const float *ab = c.acc + (size_t)bs * c.field;
    float sum = 0.f;
    for (int pz = iz; pz <= r1; ++pz) {
        float row = 0.f;
        for (int px = c0; px <= c1; ++px) row += 2.f * ab[pz * a.NX + px] / v;
        sum += row;
    }
    a.gshot[(size_t)bs * a.nz * a.nx + i] = sum;
}

CpmlArgs cpml_args(const Plan &pl, unsigned char *ws)
{
    const double dx = pl.p.dx, dz = pl.p.dz;
    CpmlArgs c;
    c.d1x = (float)(8.0 / (12.0 * dx));
    c.d2x = (float)(1.0 / (12.0 * dx));
    c.d1z = (float)(8.0 / (12.0 * dz));
    c.d2z = (float)(1.0 / (12.0 * dz));
    c.field = (size_t)pl.NZ * pl.NX;
    const size_t nbs = (size_t)pl.p.batch * pl.p.ns;
    const size_t F = align_up(nbs * c.field * 4);
    unsigned char *p = ws + pl.ws_c;
    float **fields[] = {&c.u0, &c.u1, &c.w, &c.p_x, &c.p_z, &c.z_x, &c.z_z,
                        &c.hb_x, &c.hb_z, &c.t_x, &c.t_z, &c.acc};
    for (float **f : fields) {
        *f = reinterpret_cast<float *>(p);
        p += F;
    }
    c.kap = reinterpret_cast<float *>(p);
    p += align_up((size_t)pl.p.batch * c.field * 4);
    c.rmap = reinterpret_cast<int *>(p);
    p += align_up(c.field * 4);
    c.ax = reinterpret_cast<float *>(p);
    p += align_up((size_t)pl.NX * 4);
    c.bx = reinterpret_cast<float *>(p);
    p += align_up((size_t)pl.NX * 4);
    c.az = reinterpret_cast<float *>(p);
    p += align_up((size_t)pl.NZ * 4);
    c.bz = reinterpret_cast<float *>(p);
    return c;
}

}  // namespace

size_t cpml_workspace(const Plan &pl)
{
    const size_t field = (size_t)pl.NZ * pl.NX;
    const size_t nbs = (size_t)pl.p.batch * pl.p.ns;
    return 12 * align_up(nbs * field * 4) + align_up((size_t)pl.p.batch * field * 4) +
           align_up(field * 4) + 2 * align_up((size_t)pl.NX * 4) + 2 * align_up((size_t)pl.NZ * 4);
}

cudaError_t launch_cpml(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                        cudaStream_t st)
{
    const CpmlArgs c = cpml_args(pl, ws);
    const int nbs = pl.p.batch * pl.p.ns;
    // the fields and memory variables start at rest
    cudaError_t e = cudaMemsetAsync(c.u0, 0, 12 * align_up((size_t)nbs * c.field * 4), st);
    if (e != cudaSuccess) return e;
    const double lnR = log(1.0 / pl.p.refl_R);
    const double d0x = pl.p.nb > 0 ? 3.0 * pl.p.v_ref * lnR / (2.0 * pl.p.nb * pl.p.dx) : 0.0;
    const double d0z = pl.p.nb > 0 ? 3.0 * pl.p.v_ref * lnR / (2.0 * pl.p.nb * pl.p.dz) : 0.0;
    const int cells = pl.NZ * pl.NX;
    k_cpml_setup<<<dim3((cells + 255) / 256, pl.p.batch), 256, 0, st>>>(a, c, d0x, d0z);
    k_cpml_recmap<<<(pl.p.nr + 255) / 256, 256, 0, st>>>(a, c);
    const dim3 blk(BX, BZ), grd((pl.NX + BX - 1) / BX, (pl.NZ + BZ - 1) / BZ, nbs);
    if (!adj) {
        for (int j = 0; j < pl.p.nt; ++j) {
            k_cpml_psi<<<grd, blk, 0, st>>>(a, c, j);
            if (a.snap)
                k_cpml_step<true><<<grd, blk, 0, st>>>(a, c, j);
            else
                k_cpml_step<false><<<grd, blk, 0, st>>>(a, c, j);
        }
        return cudaGetLastError();
    }
    k_cpml_adj_init<<<dim3((pl.p.nr + 127) / 128, nbs), 128, 0, st>>>(a, c);
    for (int j = pl.p.nt - 1; j >= 0; --j) {
        k_cpml_adj_a<<<grd, blk, 0, st>>>(a, c, j);
        if (j == 0) break;   // mu^0 is not needed
        k_cpml_adj_b<<<grd, blk, 0, st>>>(a, c);
        k_cpml_adj_c<<<grd, blk, 0, st>>>(a, c, j);
    }
    k_cpml_fold<<<dim3((pl.p.nz * pl.p.nx + 255) / 256, nbs), 256, 0, st>>>(a, c);
    return cudaGetLastError();
}

}  // namespace fwi
