// score_net.cu -- elementwise pieces of a convolutional score model run on the
// tensor-core convolution (conv_tc.cu): the score s(x, i) of the reverse
// diffusion (Sec. 3.4) from a noise-prediction network, s = -eps(x) /
// sqrt(1 - abar_i), and its vector-Jacobian product for Eq. chain_rule.
//   k_pack0:      X[p][0] = bf16(scale x[p]), X[p][c > 0] = 0   (fp32 -> NHWC bf16)
//   k_unpack0:    y[p] = scale Y[p][0]                          (NHWC fp32 -> fp32)
//   k_silu:       A = bf16(P / (1 + e^-P))                      (bf16 -> bf16)
//   k_silu_grad:  dP = bf16(dA silu'(P)), silu'(p) = sg (1 + p (1 - sg)), sg = 1/(1 + e^-p)
// Grid-stride loops: k_pack0 one 16-byte chunk per thread, the SiLU kernels
// eight elements per thread through 16-byte accesses where the arrays allow.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fwi_internal.cuh"
#include "silu.cuh"

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

// one thread per 16-byte chunk of X (8 channels): chunk 0 of a pixel holds
// bf16(scale x[p]) and seven zeros, the others zeros
__global__ void __launch_bounds__(kThreads)
    k_pack0(size_t npix, int C, float scale, const float *__restrict__ x,
            __nv_bfloat16 *__restrict__ X)
{
    const int per = C / 8;
    const size_t n = npix * per;
    uint4 *out = reinterpret_cast<uint4 *>(X);
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const size_t p = e / per;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (e - p * per == 0) {
            const __nv_bfloat16 h = __float2bfloat16_rn(scale * x[p]);
            v.x = (unsigned)__bfloat16_as_ushort(h);
        }
        out[e] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_unpack0(size_t npix, int C, float scale, const float *__restrict__ Y,
              float *__restrict__ y)
{
    for (size_t p = (size_t)blockIdx.x * kThreads + threadIdx.x; p < npix;
         p += (size_t)gridDim.x * kThreads)
        y[p] = scale * Y[p * C];
}


// VEC: 8 elements per thread through 16-byte accesses (n a multiple of 8,
// 16-byte aligned arrays), else one element per thread
template <bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_silu(size_t n, const __nv_bfloat16 *__restrict__ P, __nv_bfloat16 *__restrict__ A)
{
    if (VEC) {
        const uint4 *pv = reinterpret_cast<const uint4 *>(P);
        uint4 *av = reinterpret_cast<uint4 *>(A);
        for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n / 8;
             e += (size_t)gridDim.x * kThreads) {
            uint4 u = pv[e];
            __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                h[i] = __floats2bfloat162_rn(silu_of(f.x), silu_of(f.y));
            }
            av[e] = u;
        }
    } else {
        for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
             e += (size_t)gridDim.x * kThreads)
            A[e] = __float2bfloat16_rn(silu_of(__bfloat162float(P[e])));
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_silu_grad(size_t n, const __nv_bfloat16 *__restrict__ dA,
                const __nv_bfloat16 *__restrict__ P, __nv_bfloat16 *__restrict__ dP)
{
    if (VEC) {
        const uint4 *gv = reinterpret_cast<const uint4 *>(dA);
        const uint4 *pv = reinterpret_cast<const uint4 *>(P);
        uint4 *ov = reinterpret_cast<uint4 *>(dP);
        for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n / 8;
             e += (size_t)gridDim.x * kThreads) {
            uint4 g = gv[e];
            const uint4 p = pv[e];
            __nv_bfloat162 *gh = reinterpret_cast<__nv_bfloat162 *>(&g);
            const __nv_bfloat162 *ph = reinterpret_cast<const __nv_bfloat162 *>(&p);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 gf = __bfloat1622float2(gh[i]), pf = __bfloat1622float2(ph[i]);
                gh[i] = __floats2bfloat162_rn(gf.x * silu_grad_of(pf.x), gf.y * silu_grad_of(pf.y));
            }
            ov[e] = g;
        }
    } else {
        for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
             e += (size_t)gridDim.x * kThreads)
            dP[e] = __float2bfloat16_rn(__bfloat162float(dA[e]) *
                                        silu_grad_of(__bfloat162float(P[e])));
    }
}

fwi_status done(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return FWI_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

extern "C" {

fwi_status fwi_pack_channel0(long long npix, int channels, float scale, const float *x, void *X,
                             void *stream)
{
    if (npix < 1 || channels < 8 || channels % 8 != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "npix >= 1 and channels a multiple of 8");
    if (!x || !X || !aligned16(X))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x and a 16-byte aligned X are needed");
    k_pack0<<<grid_for((size_t)npix * (channels / 8)), kThreads, 0, (cudaStream_t)stream>>>(
        (size_t)npix, channels, scale, x, static_cast<__nv_bfloat16 *>(X));
    return done("fwi_pack_channel0");
}

fwi_status fwi_unpack_channel0(long long npix, int channels, float scale, const float *Y,
                               float *y, void *stream)
{
    if (npix < 1 || channels < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "npix and channels must be >= 1");
    if (!Y || !y) return fwi::record_error(FWI_ERR_INVALID_ARG, "Y and y must not be NULL");
    k_unpack0<<<grid_for((size_t)npix), kThreads, 0, (cudaStream_t)stream>>>(
        (size_t)npix, channels, scale, Y, y);
    return done("fwi_unpack_channel0");
}

fwi_status fwi_silu_bf16(long long n, const void *P, void *A, void *stream)
{
    if (n < 1 || !P || !A)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n >= 1, P and A are needed");
    if (n % 8 == 0 && aligned16(P) && aligned16(A))
        k_silu<true><<<grid_for((size_t)n / 8), kThreads, 0, (cudaStream_t)stream>>>(
            (size_t)n, static_cast<const __nv_bfloat16 *>(P), static_cast<__nv_bfloat16 *>(A));
    else
        k_silu<false><<<grid_for((size_t)n), kThreads, 0, (cudaStream_t)stream>>>(
            (size_t)n, static_cast<const __nv_bfloat16 *>(P), static_cast<__nv_bfloat16 *>(A));
    return done("fwi_silu_bf16");
}

fwi_status fwi_silu_grad_bf16(long long n, const void *dA, const void *P, void *dP, void *stream)
{
    if (n < 1 || !dA || !P || !dP)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n >= 1, dA, P and dP are needed");
    if (n % 8 == 0 && aligned16(dA) && aligned16(P) && aligned16(dP))
        k_silu_grad<true><<<grid_for((size_t)n / 8), kThreads, 0, (cudaStream_t)stream>>>(
            (size_t)n, static_cast<const __nv_bfloat16 *>(dA),
            static_cast<const __nv_bfloat16 *>(P), static_cast<__nv_bfloat16 *>(dP));
    else
        k_silu_grad<false><<<grid_for((size_t)n), kThreads, 0, (cudaStream_t)stream>>>(
            (size_t)n, static_cast<const __nv_bfloat16 *>(dA),
            static_cast<const __nv_bfloat16 *>(P), static_cast<__nv_bfloat16 *>(dP));
    return done("fwi_silu_grad_bf16");
}

}  // extern "C"
