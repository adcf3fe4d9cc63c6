// score_train.cu -- denoising score matching (Sec. 3.4, Eq. L2_rewrite) for the
// convolutional noise-prediction score model of score_net: with x_t =
// sqrt(abar) x_0 + sqrt(1 - abar) z, the conditional score is -z / sqrt(1 -
// abar), so matching s = -eps / sqrt(1 - abar) to it with the weight
// kappa(t) = 1 - abar is the regression of eps(x_t, t) on z.  Pieces:
//   k_noisy:      x_t = sqrt(abar) x_0 + sqrt(1 - abar) z
//   k_dsm:        loss = mean (eps - z)^2 (per-CTA partials added in order by
//                 k_dsm_final) and d loss / d eps = 2 (eps - z) / N
//   k_wgrad:      dW[co][ky][kx][ci] = sum_{b,p} dP[b][p][co] X[b][p + (ky-1, kx-1)][ci]
//                 (X zero outside the image), 64 x 64 (co, ci) tiles of one tap
//                 over a split of the pixels, the splits then summed in order
//                 (k_wgrad_reduce): a fixed summation order for a given split count
//   k_colsum:     db[c] = sum_p dP[p][c] (coalesced per-range partials added in
//                 order by k_colsum_final)
//   k_adam:       Adam on float32 parameters (bias-corrected moments)
//   k_wprep:      bf16 weights W and the transposed W^T[ci][ky][kx][co] =
//                 W[co][2-ky][2-kx][ci] for the backward pass, from float32
//   k_time_bias:  the per-step biases b + E phi(i) of a layer, and k_outer
//                 their gradient with respect to E, db phi(t)^T
// CUDA cores in FP32: the weight gradient reduces over every pixel of the
// batch (K = B H W), a shape the 16-byte-aligned TMA tap boxes of the
// tensor-core convolution cannot shift along.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

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

__global__ void __launch_bounds__(kThreads)
    k_noisy(size_t n, float sa, float s1, const float *__restrict__ x0, const float *__restrict__ z,
            float *__restrict__ xt)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads)
        xt[e] = fmaf(sa, x0[e], s1 * z[e]);
}

// the loss in a fixed order: CTA k sums the elements e = k 256 + t (mod G 256)
// thread-wise, then over its threads in a tree, into part[k]; k_dsm_final adds
// the G partials in order.  The gradient is elementwise.
constexpr int kLossCtas = 608;
__global__ void __launch_bounds__(kThreads)
    k_dsm(size_t n, const float *__restrict__ eps, const float *__restrict__ z,
          float *__restrict__ part, float *__restrict__ grad)
{
    __shared__ float red[kThreads];
    const float inv = 1.f / (float)n;
    float acc = 0.f;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const float d = eps[e] - z[e];
        acc = fmaf(d, d, acc);
        grad[e] = 2.f * d * inv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// thread t adds the partials t, t + 256, ... in order, then the block adds the
// 256 sums in a fixed tree
__global__ void __launch_bounds__(kThreads)
    k_dsm_final(int parts, size_t n, const float *__restrict__ part, float *__restrict__ loss)
{
    __shared__ float red[kThreads];
    float acc = 0.f;
    for (int k = threadIdx.x; k < parts; k += kThreads) acc += part[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

// CTA (tap, co tile, ci tile, pixel split): a 64 x 64 (co, ci) tile of one tap
// over one contiguous range of 32-pixel chunks; each thread keeps 4 x 4 outputs
// (co = 4 ty + i, ci = 4 tx + j).  A chunk is staged in shared memory as float
// (one 16-byte load of 8 channels per thread and operand), the next chunk's
// loads are issued before the current chunk's FMAs.  Every output is summed by
// one thread in pixel order; the splits are added in split order by
// k_wgrad_reduce.
constexpr int kWT = 64, kWP = 32, kMaxSplit = 16;

__device__ __forceinline__ void wgrad_fetch(long long p, long long npix, long long hw, int h,
                                            int w, int Cin, int Cout, int ky, int kx, int co, int ci,
                                            const __nv_bfloat16 *__restrict__ X,
                                            const __nv_bfloat16 *__restrict__ dP, uint4 &vp,
                                            uint4 &vx)
{
    vp = make_uint4(0u, 0u, 0u, 0u);
    vx = vp;
    if (p >= npix) return;
    vp = *reinterpret_cast<const uint4 *>(dP + p * Cout + co);
    const long long b = p / hw;
    const int r = (int)(p - b * hw);
    const int y = r / w + ky - 1, x = r % w + kx - 1;
    if (y >= 0 && y < h && x >= 0 && x < w)
        vx = *reinterpret_cast<const uint4 *>(X + ((b * h + y) * (long long)w + x) * Cin + ci);
}

__device__ __forceinline__ void stage8(float *dst, uint4 v)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
    float4 lo, hi;
    float2 f;
    f = __bfloat1622float2(h[0]); lo.x = f.x; lo.y = f.y;
    f = __bfloat1622float2(h[1]); lo.z = f.x; lo.w = f.y;
    f = __bfloat1622float2(h[2]); hi.x = f.x; hi.y = f.y;
    f = __bfloat1622float2(h[3]); hi.z = f.x; hi.w = f.y;
    reinterpret_cast<float4 *>(dst)[0] = lo;
    reinterpret_cast<float4 *>(dst)[1] = hi;
}

__global__ void __launch_bounds__(kThreads)
    k_wgrad(int n, int h, int w, int Cin, int Cout, long long chunks_per_split,
            const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ dP,
            float *__restrict__ out)
{
    __shared__ __align__(16) float sP[kWP][kWT];
    __shared__ __align__(16) float sX[kWP][kWT];
    const int ci_tiles = Cin / kWT;
    int t = blockIdx.x;
    const int tap = t % 9;
    t /= 9;
    const int ci0 = (t % ci_tiles) * kWT, co0 = (t / ci_tiles) * kWT;
    const int ky = tap / 3, kx = tap % 3;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int lp = threadIdx.x / 8, lq = (threadIdx.x % 8) * 8;   // loader: pixel, 8 channels
    const long long npix = (long long)n * h * w, hw = (long long)h * w;
    const long long nchunks = (npix + kWP - 1) / kWP;
    const long long c0 = (long long)blockIdx.y * chunks_per_split;
    const long long c1 = c0 + chunks_per_split < nchunks ? c0 + chunks_per_split : nchunks;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    uint4 vp, vx;
    if (c0 < c1)
        wgrad_fetch(c0 * kWP + lp, npix, hw, h, w, Cin, Cout, ky, kx, co0 + lq, ci0 + lq, X, dP, vp,
                    vx);
    for (long long ch = c0; ch < c1; ++ch) {
        stage8(&sP[lp][lq], vp);
        stage8(&sX[lp][lq], vx);
        __syncthreads();
        if (ch + 1 < c1)
            wgrad_fetch((ch + 1) * kWP + lp, npix, hw, h, w, Cin, Cout, ky, kx, co0 + lq, ci0 + lq,
                        X, dP, vp, vx);
#pragma unroll 8
        for (int pl = 0; pl < kWP; ++pl) {
            const float4 a = *reinterpret_cast<const float4 *>(&sP[pl][4 * ty]);
            const float4 b = *reinterpret_cast<const float4 *>(&sX[pl][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *o = out + (size_t)blockIdx.y * 9 * Cin * Cout;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + 4 * ty + i;
        *reinterpret_cast<float4 *>(o + ((size_t)co * 9 + tap) * Cin + ci0 + 4 * tx) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
}

// dW[e] = sum_s work[s][e], s in order
__global__ void __launch_bounds__(kThreads)
    k_wgrad_reduce(size_t n, int splits, const float *__restrict__ work, float *__restrict__ dW)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        float s = work[e];
        for (int k = 1; k < splits; ++k) s += work[(size_t)k * n + e];
        dW[e] = s;
    }
}

// db[c] = sum_p dP[p][c]: CTA k sums the pixels of range k, its threads laid
// out as `lanes` pixel lanes x channels (consecutive threads read consecutive
// channels of one pixel), the lanes then added in order into part[k][c];
// k_colsum_final adds the ranges in order.
__global__ void __launch_bounds__(kThreads)
    k_colsum(long long npix, int C, int lanes, long long per, const __nv_bfloat16 *__restrict__ dP,
             float *__restrict__ part)
{
    __shared__ float red[kThreads];
    const int lane = threadIdx.x / C, c = threadIdx.x % C;
    const long long p0 = (long long)blockIdx.x * per;
    const long long p1 = p0 + per < npix ? p0 + per : npix;
    for (int c0 = 0; c0 < C; c0 += kThreads) {
        // C > 256: one lane, channel blocks of 256
        const int cc = lanes > 1 ? c : c0 + (int)threadIdx.x;
        float acc = 0.f;
        if (lane < lanes && cc < C)
            for (long long p = p0 + lane; p < p1; p += lanes) acc += __bfloat162float(dP[p * C + cc]);
        red[threadIdx.x] = acc;
        __syncthreads();
        if (lanes > 1) {
            if ((int)threadIdx.x < C) {
                float s2 = red[threadIdx.x];
                for (int l = 1; l < lanes; ++l) s2 += red[l * C + threadIdx.x];
                part[(size_t)blockIdx.x * C + threadIdx.x] = s2;
            }
        } else if (cc < C) {
            part[(size_t)blockIdx.x * C + cc] = red[threadIdx.x];
        }
        __syncthreads();
        if (lanes > 1) break;
    }
}

// CTA: 32 channels x 8 groups; group g adds the ranges g, g + 8, ... in order,
// then the 8 group sums are added in order
// the same with 16-byte loads: a thread sums 8 channels (C / 8 threads per
// pixel, lanes = 256 / (C / 8) pixel lanes), the lanes then added in order
__global__ void __launch_bounds__(kThreads)
    k_colsum8(long long npix, int C, int lanes, long long per, const __nv_bfloat16 *__restrict__ dP,
              float *__restrict__ part)
{
    __shared__ float red[kThreads * 8];
    const int tpp = C / 8;
    const int lane = threadIdx.x / tpp, c8 = (threadIdx.x % tpp) * 8;
    const long long p0 = (long long)blockIdx.x * per;
    const long long p1 = p0 + per < npix ? p0 + per : npix;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long p = p0 + lane; p < p1; p += lanes) {
        const uint4 u = *reinterpret_cast<const uint4 *>(dP + p * C + c8);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(h[i]);
            acc[2 * i] += f.x;
            acc[2 * i + 1] += f.y;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) red[lane * C + c8 + i] = acc[i];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += kThreads) {
        float s2 = red[c];
        for (int l = 1; l < lanes; ++l) s2 += red[l * C + c];
        part[(size_t)blockIdx.x * C + c] = s2;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_colsum_final(int parts, int C, const float *__restrict__ part, float *__restrict__ db)
{
    __shared__ float red[8][32];
    const int g = threadIdx.x / 32, c = blockIdx.x * 32 + threadIdx.x % 32;
    float acc = 0.f;
    if (c < C)
        for (int k = g; k < parts; k += 8) acc += part[(size_t)k * C + c];
    red[g][threadIdx.x % 32] = acc;
    __syncthreads();
    if (g == 0 && c < C) {
        float s2 = red[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) s2 += red[k][threadIdx.x];
        db[c] = s2;
    }
}

// 1 - b1 and 1 - b2 formed in double on the host: 1 - (float)0.999 in float
// would be off by 1.3e-5 relative
struct AdamF {
    float lr, b1, b2, omb1, omb2, eps, c1, c2;   // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

__global__ void __launch_bounds__(kThreads)
    k_adam(size_t n, AdamF k, float *__restrict__ p, const float *__restrict__ g,
           float *__restrict__ m, float *__restrict__ v)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const float ge = g[e];
        const float me = fmaf(k.b1, m[e], k.omb1 * ge);
        const float ve = fmaf(k.b2, v[e], k.omb2 * ge * ge);
        m[e] = me;
        v[e] = ve;
        p[e] -= k.lr * (me * k.c1) / (sqrtf(ve * k.c2) + k.eps);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_wprep(int C, int Cin, const float *__restrict__ W, __nv_bfloat16 *__restrict__ Wb,
            __nv_bfloat16 *__restrict__ WTb)
{
    const size_t n = (size_t)C * 9 * Cin;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const int ci = (int)(e % Cin);
        const int tap = (int)((e / Cin) % 9);
        const int co = (int)(e / ((size_t)Cin * 9));
        const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
        Wb[e] = b;
        // W^T[ci][8 - tap][co] = W[co][tap][ci]
        WTb[((size_t)ci * 9 + (8 - tap)) * C + co] = b;
    }
}

// out[i][c] = b[c] + sum_k E[c][k] phi[i][k]: the per-step biases of a layer
__global__ void __launch_bounds__(kThreads)
    k_time_bias(int nsteps, int C, int dim, const float *__restrict__ b, const float *__restrict__ E,
                const float *__restrict__ phi, float *__restrict__ out)
{
    const size_t n = (size_t)nsteps * C;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const int i = (int)(e / C), c = (int)(e % C);
        float s = b[c];
        for (int k = 0; k < dim; ++k) s = fmaf(E[(size_t)c * dim + k], phi[(size_t)i * dim + k], s);
        out[e] = s;
    }
}

// dE[c][k] = db[c] phi[k]
__global__ void __launch_bounds__(kThreads)
    k_outer(int C, int dim, const float *__restrict__ db, const float *__restrict__ phi,
            float *__restrict__ dE)
{
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < C * dim; e += gridDim.x * kThreads)
        dE[e] = db[e / dim] * phi[e % dim];
}

fwi_status done(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_dsm_noisy(long long n, double abar, const float *x0, const float *z, float *xt,
                         void *stream)
{
    if (n < 1 || !(abar > 0.0 && abar < 1.0) || !x0 || !z || !xt)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n >= 1, 0 < abar < 1 and arrays needed");
    k_noisy<<<grid_for((size_t)n), kThreads, 0, (cudaStream_t)stream>>>(
        (size_t)n, (float)std::sqrt(abar), (float)std::sqrt(1.0 - abar), x0, z, xt);
    return done("fwi_dsm_noisy");
}

fwi_status fwi_dsm_loss(long long n, const float *eps, const float *z, float *loss, float *grad,
                        float *work, long long work_floats, void *stream)
{
    if (n < 1 || !eps || !z || !loss || !grad)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n >= 1 and arrays needed");
    cudaStream_t st = (cudaStream_t)stream;
    // without room for the partials: one CTA, its partial written to loss
    long long g = work ? (work_floats < kLossCtas ? work_floats : kLossCtas) : 1;
    const long long need = ((long long)n + kThreads - 1) / kThreads;
    if (g > need) g = need;
    if (g < 1) g = 1;
    float *part = g > 1 ? work : loss;
    k_dsm<<<(unsigned)g, kThreads, 0, st>>>((size_t)n, eps, z, part, grad);
    k_dsm_final<<<1, kThreads, 0, st>>>((int)g, (size_t)n, part, loss);
    return done("fwi_dsm_loss");
}

int fwi_conv3x3_wgrad_splits(int n, int h, int w, int cin, int cout, long long work_floats)
{
    if (n < 1 || h < 1 || w < 1 || cin < kWT || cin % kWT != 0 || cout < kWT || cout % kWT != 0)
        return 0;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ctas = 9LL * (cin / kWT) * (cout / kWT);
    const long long nchunks = ((long long)n * h * w + kWP - 1) / kWP;
    long long s = (4LL * sms + ctas - 1) / ctas;       // about 4 CTAs per SM
    if (s > kMaxSplit) s = kMaxSplit;
    if (s > nchunks) s = nchunks;
    const long long fit = work_floats / (9LL * cin * cout);
    if (s > fit) s = fit;
    return s < 1 ? 1 : (int)s;
}

fwi_status fwi_conv3x3_wgrad(int n, int h, int w, int cin, int cout, const void *X, const void *dP,
                             float *dW, float *work, long long work_floats, void *stream)
{
    if (n < 1 || h < 1 || w < 1 || cin < kWT || cin % kWT != 0 || cout < kWT || cout % kWT != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "n, h, w >= 1 and cin, cout multiples of 64");
    if (!X || !dP || !dW) return fwi::record_error(FWI_ERR_INVALID_ARG, "X, dP and dW are needed");
    if (((uintptr_t)X & 15) || ((uintptr_t)dP & 15) || ((uintptr_t)dW & 15) ||
        ((uintptr_t)work & 15))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "X, dP, dW and work must be 16-byte aligned");
    const int splits = fwi_conv3x3_wgrad_splits(n, h, w, cin, cout, work ? work_floats : 0);
    const long long nchunks = ((long long)n * h * w + kWP - 1) / kWP;
    const long long per = (nchunks + splits - 1) / splits;
    const dim3 grid(9 * (cin / kWT) * (cout / kWT), splits);
    float *out = splits > 1 ? work : dW;
    k_wgrad<<<grid, kThreads, 0, (cudaStream_t)stream>>>(
        n, h, w, cin, cout, per, static_cast<const __nv_bfloat16 *>(X),
        static_cast<const __nv_bfloat16 *>(dP), out);
    if (splits > 1) {
        const size_t nw = (size_t)9 * cin * cout;
        k_wgrad_reduce<<<grid_for(nw), kThreads, 0, (cudaStream_t)stream>>>(nw, splits, work, dW);
    }
    return done("fwi_conv3x3_wgrad");
}

fwi_status fwi_channel_sum(long long npix, int channels, const void *dP, float *db, float *work,
                           long long work_floats, void *stream)
{
    if (npix < 1 || channels < 1 || !dP || !db)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "npix, channels >= 1 and arrays needed");
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int lanes = channels <= kThreads && kThreads % channels == 0 ? kThreads / channels : 1;
    long long parts = work ? work_floats / channels : 0;
    if (parts > 4LL * sms) parts = 4LL * sms;
    if (parts > npix) parts = npix;
    float *part = work;
    if (parts < 2) {
        // one range: its partial is the result
        parts = 1;
        part = db;
    }
    const long long per = (npix + parts - 1) / parts;
    cudaStream_t st = (cudaStream_t)stream;
    // 16-byte loads when a pixel's channels split into 8-channel groups that
    // tile the block
    const bool vec = channels % 8 == 0 && channels / 8 <= kThreads &&
                     kThreads % (channels / 8) == 0 && ((uintptr_t)dP & 15) == 0;
    if (vec)
        k_colsum8<<<(unsigned)parts, kThreads, 0, st>>>(npix, channels, kThreads / (channels / 8),
                                                       per, static_cast<const __nv_bfloat16 *>(dP),
                                                       part);
    else
        k_colsum<<<(unsigned)parts, kThreads, 0, st>>>(npix, channels, lanes, per,
                                                      static_cast<const __nv_bfloat16 *>(dP), part);
    if (parts > 1)
        k_colsum_final<<<(unsigned)((channels + 31) / 32), kThreads, 0, st>>>((int)parts, channels,
                                                                              part, db);
    return done("fwi_channel_sum");
}

fwi_status fwi_adam_step(long long n, double lr, double beta1, double beta2, double eps, int step,
                         float *param, const float *grad, float *m, float *v, void *stream)
{
    if (n < 1 || step < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
        !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !param || !grad || !m || !v)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "invalid Adam arguments");
    AdamF k{(float)lr, (float)beta1, (float)beta2, (float)(1.0 - beta1), (float)(1.0 - beta2),
            (float)eps,
            (float)(1.0 / (1.0 - std::pow(beta1, step))),
            (float)(1.0 / (1.0 - std::pow(beta2, step)))};
    k_adam<<<grid_for((size_t)n), kThreads, 0, (cudaStream_t)stream>>>((size_t)n, k, param, grad,
                                                                        m, v);
    return done("fwi_adam_step");
}

fwi_status fwi_conv3x3_weights_prep(int cout, int cin, const float *W, void *Wb, void *WTb,
                                    void *stream)
{
    if (cout < 1 || cin < 1 || !W || !Wb || !WTb)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "cout, cin >= 1 and arrays needed");
    k_wprep<<<grid_for((size_t)cout * 9 * cin), kThreads, 0, (cudaStream_t)stream>>>(
        cout, cin, W, static_cast<__nv_bfloat16 *>(Wb), static_cast<__nv_bfloat16 *>(WTb));
    return done("fwi_conv3x3_weights_prep");
}

fwi_status fwi_time_bias(int nsteps, int channels, int dim, const float *b, const float *E,
                         const float *phi, float *out, void *stream)
{
    if (nsteps < 1 || channels < 1 || dim < 1 || !b || !E || !phi || !out)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "sizes >= 1 and arrays needed");
    k_time_bias<<<grid_for((size_t)nsteps * channels), kThreads, 0, (cudaStream_t)stream>>>(
        nsteps, channels, dim, b, E, phi, out);
    return done("fwi_time_bias");
}

fwi_status fwi_time_bias_grad(int channels, int dim, const float *db, const float *phi, float *dE,
                              void *stream)
{
    if (channels < 1 || dim < 1 || !db || !phi || !dE)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "sizes >= 1 and arrays needed");
    k_outer<<<grid_for((size_t)channels * dim), kThreads, 0, (cudaStream_t)stream>>>(
        channels, dim, db, phi, dE);
    return done("fwi_time_bias_grad");
}

}  // extern "C"
