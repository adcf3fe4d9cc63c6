// baselines.cu -- the data potential of the DPS baseline, the TV subgradient
// of the TV-regularised baselines, and the reconstruction measures (Sec. 4.2,
// 6.3).  One CTA per instance, fixed reduction orders (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int NT_B = 1024;
constexpr unsigned FULL = 0xffffffffu;

__device__ float block_sum(float v, float *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float u = red[lane];   // NT_B / 32 == 32 warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(FULL, u, o);
        if (lane == 0) red[32] = u;
    }
    __syncthreads();
    return red[32];
}

// J[b] = (1/2) sum (d_syn - d_obs)^2 / sigma^2, adj = (d_syn - d_obs) / sigma^2
__global__ void __launch_bounds__(NT_B) k_l2_misfit(size_t n, float inv_s2,
                                                    const float *__restrict__ dobs,
                                                    const float *__restrict__ dsyn,
                                                    float *__restrict__ J, float *__restrict__ adj)
{
    __shared__ float red[33];
    const size_t off = (size_t)blockIdx.x * n;
    float part = 0.f;
    for (size_t i = threadIdx.x; i < n; i += NT_B) {
        const float r = dsyn[off + i] - dobs[off + i];
        part = fmaf(0.5f * r, r, part);
        if (adj) adj[off + i] = r * inv_s2;
    }
    const float s = block_sum(part, red);
    if (threadIdx.x == 0) J[blockIdx.x] = s * inv_s2;
}

// TV(v / unit) = (1/N_g) sum |forward differences| / unit (a difference leaving
// the grid counts as 0) and h = g + alpha dTV/dv: every difference d between
// a cell and its right (lower) neighbour adds alpha sign(d) / (N_g unit) to
// the neighbour and subtracts it from the cell (sign(0) = 0).
__global__ void __launch_bounds__(NT_B) k_tv_grad(int nz, int nx, float coef, float inv_unit,
                                                  const float *__restrict__ v,
                                                  const float *__restrict__ g,
                                                  float *__restrict__ h, float *__restrict__ tv)
{
    __shared__ float red[33];
    const int n = nz * nx;
    const size_t off = (size_t)blockIdx.x * n;
    const float *vb = v + off;
    float part = 0.f;
    for (int i = threadIdx.x; i < n; i += NT_B) {
        const int iz = i / nx, ix = i - (i / nx) * nx;
        const float c = vb[i];
        float s = 0.f;
        if (ix + 1 < nx) {
            const float d = vb[i + 1] - c;
            part += fabsf(d);
            s -= (d > 0.f) - (d < 0.f);
        }
        if (iz + 1 < nz) {
            const float d = vb[i + nx] - c;
            part += fabsf(d);
            s -= (d > 0.f) - (d < 0.f);
        }
        if (ix > 0) {
            const float d = c - vb[i - 1];
            s += (d > 0.f) - (d < 0.f);
        }
        if (iz > 0) {
            const float d = c - vb[i - nx];
            s += (d > 0.f) - (d < 0.f);
        }
        h[off + i] = (g ? g[off + i] : 0.f) + coef * s;
    }
    const float t = block_sum(part, red);
    if (threadIdx.x == 0 && tv) tv[blockIdx.x] = t * inv_unit / (float)n;
}

// relative l2 error, PSNR, SSIM (11 x 11 Gaussian window, sigma 1.5, every
// window inside the grid, two-pass weighted moments)
__global__ void __launch_bounds__(NT_B) k_image_metrics(int nz, int nx, float R,
                                                        const float *__restrict__ vt,
                                                        const float *__restrict__ vr,
                                                        float *__restrict__ out)
{
    __shared__ float red[33];
    __shared__ float w[121];
    const int n = nz * nx;
    const size_t off = (size_t)blockIdx.x * n;
    const float *t = vt + off, *r = vr + off;
    if (threadIdx.x < 121) {
        const int a = threadIdx.x / 11 - 5, b = threadIdx.x % 11 - 5;
        w[threadIdx.x] = expf(-(float)(a * a + b * b) / (2.f * 1.5f * 1.5f));
    }
    __syncthreads();
    float ws = 0.f;
    for (int k = 0; k < 121; ++k) ws += w[k];   // every thread, same order
    float se = 0.f, st = 0.f;
    for (int i = threadIdx.x; i < n; i += NT_B) {
        const float e = t[i] - r[i];
        se = fmaf(e, e, se);
        st = fmaf(t[i], t[i], st);
    }
    se = block_sum(se, red);
    st = block_sum(st, red);
    const float C1 = (0.01f * R) * (0.01f * R), C2 = (0.03f * R) * (0.03f * R);
    const int wz = nz - 10, wx = nx - 10;
    float ss = 0.f;
    for (int q = threadIdx.x; q < (wz > 0 && wx > 0 ? wz * wx : 0); q += NT_B) {
        const int i = q / wx, j = q - (q / wx) * wx;
        float mt = 0.f, mr = 0.f;
        for (int a = 0; a < 11; ++a)
            for (int b = 0; b < 11; ++b) {
                const float ww = w[a * 11 + b] / ws;
                mt = fmaf(ww, t[(i + a) * nx + j + b], mt);
                mr = fmaf(ww, r[(i + a) * nx + j + b], mr);
            }
        float vtt = 0.f, vrr = 0.f, vtr = 0.f;
        for (int a = 0; a < 11; ++a)
            for (int b = 0; b < 11; ++b) {
                const float ww = w[a * 11 + b] / ws;
                const float dt = t[(i + a) * nx + j + b] - mt, dr = r[(i + a) * nx + j + b] - mr;
                vtt = fmaf(ww * dt, dt, vtt);
                vrr = fmaf(ww * dr, dr, vrr);
                vtr = fmaf(ww * dt, dr, vtr);
            }
        ss += (2.f * mt * mr + C1) * (2.f * vtr + C2) /
              ((mt * mt + mr * mr + C1) * (vtt + vrr + C2));
    }
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) {
        out[3 * blockIdx.x + 0] = sqrtf(se) / sqrtf(st);
        out[3 * blockIdx.x + 1] = 10.f * log10f(R * R / (se / (float)n));
        out[3 * blockIdx.x + 2] = (wz > 0 && wx > 0) ? ss / (float)(wz * wx) : NAN;
    }
}

}  // namespace

}  // namespace fwi

extern "C" {

FWI_API fwi_status fwi_l2_misfit(const fwi_plan *plan, const float *d_obs, const float *d_syn,
                                 double sigma, float *J, float *adj_src, void *stream)
{
    if (!plan || !d_obs || !d_syn || !J)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "plan, d_obs, d_syn and J must not be NULL");
    if (!(sigma > 0.0) || !std::isfinite(sigma))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "sigma must be finite and > 0");
    const fwi::Plan &pl = *reinterpret_cast<const fwi::Plan *>(plan);
    const size_t n = (size_t)pl.p.ns * pl.p.nr * pl.p.nt;
    fwi::k_l2_misfit<<<pl.p.batch, fwi::NT_B, 0, (cudaStream_t)stream>>>(
        n, (float)(1.0 / (sigma * sigma)), d_obs, d_syn, J, adj_src);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_l2_misfit launch: %s", cudaGetErrorString(e));
    return FWI_OK;
}

FWI_API fwi_status fwi_tv_grad(int batch, int nz, int nx, double alpha, double unit,
                               const float *v, const float *g, float *h, float *tv, void *stream)
{
    if (batch < 1 || nz < 1 || nx < 1 || !v || !h)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "need batch, nz, nx >= 1 and v, h");
    if (!std::isfinite(alpha) || !(unit > 0.0) || !std::isfinite(unit))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "alpha must be finite and unit > 0");
    if ((size_t)nz * nx > (size_t)1 << 30)
        return fwi::record_error(FWI_ERR_UNSUPPORTED, "grid too large");
    const double coef = alpha / ((double)nz * nx * unit);
    fwi::k_tv_grad<<<batch, fwi::NT_B, 0, (cudaStream_t)stream>>>(nz, nx, (float)coef,
                                                                  (float)(1.0 / unit), v, g, h, tv);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_tv_grad launch: %s", cudaGetErrorString(e));
    return FWI_OK;
}

FWI_API fwi_status fwi_image_metrics(int batch, int nz, int nx, double data_range,
                                     const float *v_true, const float *v_rec, float *out,
                                     void *stream)
{
    if (batch < 1 || nz < 1 || nx < 1 || !v_true || !v_rec || !out)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "need batch, nz, nx >= 1 and all arrays");
    if (!(data_range > 0.0) || !std::isfinite(data_range))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "data_range must be finite and > 0");
    if ((size_t)nz * nx > (size_t)1 << 30)
        return fwi::record_error(FWI_ERR_UNSUPPORTED, "grid too large");
    fwi::k_image_metrics<<<batch, fwi::NT_B, 0, (cudaStream_t)stream>>>(nz, nx, (float)data_range,
                                                                        v_true, v_rec, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_image_metrics launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

}  // extern "C"
