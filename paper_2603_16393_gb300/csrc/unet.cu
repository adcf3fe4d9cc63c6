// unet.cu -- the resampling steps of a U-Net score network (the score model of
// Sec. 6 is a U-Net): between levels the activations are halved by 2 x 2
// average pooling and doubled back by nearest-neighbour upsampling, and the
// decoder adds the encoder's activations of its level (additive skips).
// NHWC bf16, FP32 arithmetic, one 8-channel (16-byte) chunk per thread:
//   k_pool2: y[b][I][J][c] = s * sum of x[b][i][j][c] over the block i in {2I, 2I+1},
//            j in {2J, 2J+1} inside the h x w image; s = 1 / (cells in the block)
//            (mode 0: the mean) or 1 (mode 1: the sum, the adjoint of mode-0 upsampling)
//   k_up2:   y[b][i][j][c] = s * x[b][i/2][j/2][c] for i < ho, j < wo; s = 1 (mode 0)
//            or 1 / (cells of block (i/2, j/2) inside ho x wo) (mode 1: the adjoint of
//            mean pooling)
//   k_add:   z = x + y
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace {

constexpr int kThreads = 256;

unsigned grid_for(size_t n)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n + kThreads - 1) / kThreads;
    const size_t cap = (size_t)sms * 8;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

__device__ __forceinline__ void add8(float (&acc)[8], uint4 u)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        acc[2 * i] += f.x;
        acc[2 * i + 1] += f.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8], float s)
{
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(s * v[2 * i], s * v[2 * i + 1]);
    return u;
}

__global__ void __launch_bounds__(kThreads)
    k_pool2(int n, int h, int w, int C, int mode, const uint4 *__restrict__ x, uint4 *__restrict__ y)
{
    const int hc = (h + 1) / 2, wc = (w + 1) / 2, cg = C / 8;
    const size_t total = (size_t)n * hc * wc * cg;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int g = (int)(e % cg);
        const size_t pix = e / cg;
        const int J = (int)(pix % wc), I = (int)((pix / wc) % hc);
        const size_t b = pix / ((size_t)wc * hc);
        const int i1 = min(2 * I + 2, h), j1 = min(2 * J + 2, w);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = 2 * I; i < i1; ++i)
            for (int j = 2 * J; j < j1; ++j) add8(acc, x[((b * h + i) * w + j) * cg + g]);
        const float s = mode == 0 ? 1.f / (float)((i1 - 2 * I) * (j1 - 2 * J)) : 1.f;
        y[e] = pack8(acc, s);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_up2(int n, int ho, int wo, int C, int mode, const uint4 *__restrict__ x, uint4 *__restrict__ y)
{
    const int hc = (ho + 1) / 2, wc = (wo + 1) / 2, cg = C / 8;
    const size_t total = (size_t)n * ho * wo * cg;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int g = (int)(e % cg);
        const size_t pix = e / cg;
        const int j = (int)(pix % wo), i = (int)((pix / wo) % ho);
        const size_t b = pix / ((size_t)wo * ho);
        const int I = i / 2, J = j / 2;
        const uint4 u = x[((b * hc + I) * wc + J) * cg + g];
        if (mode == 0) {
            y[e] = u;
        } else {
            const int cnt = (min(2 * I + 2, ho) - 2 * I) * (min(2 * J + 2, wo) - 2 * J);
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            add8(v, u);
            y[e] = pack8(v, 1.f / (float)cnt);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
    k_add(size_t n8, const uint4 *__restrict__ x, const uint4 *__restrict__ y, uint4 *__restrict__ z)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n8;
         e += (size_t)gridDim.x * kThreads) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        add8(v, x[e]);
        add8(v, y[e]);
        z[e] = pack8(v, 1.f);
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

fwi_status done(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_pool2_bf16(int n, int h, int w, int channels, int mode, const void *x, void *y,
                          void *stream)
{
    if (n < 1 || h < 1 || w < 1 || channels < 8 || channels % 8 != 0 || (mode != 0 && mode != 1))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "n, h, w >= 1, channels a multiple of 8, mode 0 or 1");
    if (!x || !y || !aligned16(x) || !aligned16(y))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    const size_t total = (size_t)n * ((h + 1) / 2) * ((w + 1) / 2) * (channels / 8);
    k_pool2<<<grid_for(total), kThreads, 0, (cudaStream_t)stream>>>(
        n, h, w, channels, mode, static_cast<const uint4 *>(x), static_cast<uint4 *>(y));
    return done("fwi_pool2_bf16");
}

fwi_status fwi_up2_bf16(int n, int ho, int wo, int channels, int mode, const void *x, void *y,
                        void *stream)
{
    if (n < 1 || ho < 1 || wo < 1 || channels < 8 || channels % 8 != 0 || (mode != 0 && mode != 1))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "n, ho, wo >= 1, channels a multiple of 8, mode 0 or 1");
    if (!x || !y || !aligned16(x) || !aligned16(y))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    const size_t total = (size_t)n * ho * wo * (channels / 8);
    k_up2<<<grid_for(total), kThreads, 0, (cudaStream_t)stream>>>(
        n, ho, wo, channels, mode, static_cast<const uint4 *>(x), static_cast<uint4 *>(y));
    return done("fwi_up2_bf16");
}

fwi_status fwi_add_bf16(long long count, const void *x, const void *y, void *z, void *stream)
{
    if (count < 8 || count % 8 != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "count must be a positive multiple of 8");
    if (!x || !y || !z || !aligned16(x) || !aligned16(y) || !aligned16(z))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x, y and z must be 16-byte aligned");
    k_add<<<grid_for((size_t)count / 8), kThreads, 0, (cudaStream_t)stream>>>(
        (size_t)count / 8, static_cast<const uint4 *>(x), static_cast<const uint4 *>(y),
        static_cast<uint4 *>(z));
    return done("fwi_add_bf16");
}

}  // extern "C"
