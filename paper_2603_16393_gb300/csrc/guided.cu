// guided.cu -- preconditioned guided update of Algorithm 2 (Sec. 5.2),
// one CTA per instance:
//   TV    = (1/N_g) sum (|v0hat[z][x+1]-v0hat[z][x]| + |v0hat[z+1][x]-v0hat[z][x]|)  (Eq. tv)
//   rho   = rho0 exp(-(TV - tau)_+ / c)                                             (Eq. rho)
//   kappa = ((||g||_inf + eps) / (|g| + eps))^gamma, clipped if kmin < kmax         (Eq. kappa)
//   v_out = v' - rho kappa h                                                        (Eq. precond_step)
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int NT_G = 1024;
constexpr unsigned FULL = 0xffffffffu;

template <bool MAX>
__device__ float block_reduce_g(float v, float *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(FULL, v, o);
        v = MAX ? fmaxf(v, u) : v + u;
    }
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float u = red[lane];   // NT_G / 32 == 32 warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float t = __shfl_xor_sync(FULL, u, o);
            u = MAX ? fmaxf(u, t) : u + t;
        }
        if (lane == 0) red[32] = u;
    }
    __syncthreads();
    return red[32];
}

struct GuideF {
    float rho0, c, tau, gamma, eps, kappa_min, kappa_max;
    float inv_unit, unit, unit2;   // normalised-space unit and its powers
};

__global__ void __launch_bounds__(NT_G) k_guided(int nz, int nx, GuideF gp,
                                                 const float *vprime,
                                                 const float *__restrict__ v0hat,
                                                 const float *__restrict__ g,
                                                 const float *__restrict__ h, float *vout,
                                                 float *__restrict__ rho_out)
{
    __shared__ float red[33];
    const int n = nz * nx;
    const size_t off = (size_t)blockIdx.x * n;
    const float *v0 = v0hat + off, *gb = g + off;
    float tv = 0.f, gmax = 0.f;
    for (int i = threadIdx.x; i < n; i += NT_G) {
        const int iz = i / nx, ix = i - (i / nx) * nx;
        const float c = v0[i];
        if (ix + 1 < nx) tv += fabsf(v0[i + 1] - c);
        if (iz + 1 < nz) tv += fabsf(v0[i + nx] - c);
        gmax = fmaxf(gmax, fabsf(gb[i]));
    }
    tv = block_reduce_g<false>(tv, red) / ((float)nz * (float)nx) * gp.inv_unit;
    gmax = block_reduce_g<true>(gmax, red) * gp.unit;
    const float rho = gp.rho0 * expf(-fmaxf(tv - gp.tau, 0.f) / gp.c);
    const bool clip = gp.kappa_min < gp.kappa_max;
    for (int i = threadIdx.x; i < n; i += NT_G) {
        float kap = powf((gmax + gp.eps) / (fabsf(gb[i]) * gp.unit + gp.eps), gp.gamma);
        if (clip) kap = fminf(fmaxf(kap, gp.kappa_min), gp.kappa_max);
        vout[off + i] = vprime[off + i] - rho * kap * (gp.unit2 * h[off + i]);
    }
    if (threadIdx.x == 0 && rho_out) rho_out[blockIdx.x] = rho;
}

}  // namespace

cudaError_t launch_guided(int B, int nz, int nx, const fwi_guide_params &gp, const float *vprime,
                          const float *v0hat, const float *g, const float *h, float *vout,
                          float *rho, cudaStream_t st)
{
    const GuideF gf = {(float)gp.rho0, (float)gp.c, (float)gp.tau, (float)gp.gamma,
                       (float)gp.eps, (float)gp.kappa_min, (float)gp.kappa_max,
                       (float)(1.0 / gp.unit), (float)gp.unit, (float)(gp.unit * gp.unit)};
    k_guided<<<B, NT_G, 0, st>>>(nz, nx, gf, vprime, v0hat, g, h, vout, rho);
    return cudaGetLastError();
}

}  // namespace fwi
