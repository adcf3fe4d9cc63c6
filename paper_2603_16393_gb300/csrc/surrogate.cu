// surrogate.cu -- the data-side steps of the learned forward surrogate, a
// convolutional encoder-decoder from a velocity model to the seismograms of
// the FD solver (the surrogate route to cheaper guidance of Sec. 7, used in
// the early reverse steps of Algorithm 2).  Its six convolutions run on the
// tensor-core convolution (fwi_conv3x3_bf16) with SiLU, skip and training
// kernels shared with the score networks; this file holds what is particular
// to it:
//
//   layout   model b is column b mod m of image b / m: an image is nx pixels
//            high (the model's columns x) and m pixels wide (m models side by
//            side); the convolutions keep their horizontal taps at zero, so
//            the models never see each other and each pixel couples only to
//            x - 1, x, x + 1 of its own model
//   k_pack   X0[img][x][col][c] = bf16(in_scale v[b][c][x] + in_shift) for
//            c < nz, bf16(G[x][c]) (geometry channels) above; columns past
//            the last model are zero
//   k_unpack dv[b][z][x] = in_scale dX[img][x][col][z] (the input gradient)
//   k_traces d[b][s][r][t] = amp sign(y) (e^|y| - 1), y = Y[img][rec_ix[r]][col][s nt + t]
//   k_outgrad dY = bf16(scale adj[b][s][r][t] amp e^|y|) at the receivers'
//            columns and channels s nt + t, 0 elsewhere: the transpose of the
//            trace map's derivative
//   k_target Yt = sign(d) log(1 + |d| / amp) there, 0 elsewhere
//   k_loss   mean (Y - Yt)^2 (per-CTA partials added in order) and
//            dY = bf16(2 (Y - Yt) / N)
//   k_pool_h, k_up_h  mean pooling of row pairs and nearest upsampling along
//            the image (mode 1: their adjoints, sum pooling and division by
//            the block's rows)
//   k_wprep3 bf16 3 x 3 weights with zero horizontal taps, and their
//            transpose W^T[ci][ky][kx][co] = W[co][2-ky][2-kx][ci], from the
//            three-tap float32 weights W3[co][ky][ci]
//   k_wcentre dW3[co][ky][ci] = dW[co][ky][1][ci] (the taps the network has)
//   k_rel_err err[b] = ||g_b - r_b|| / ||r_b|| per model (the FD check's
//            measure of the surrogate's gradient), sums in double, one CTA a
//            model, a fixed order
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "fwi_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kLossCtas = 608;

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
    k_pack(int nmod, int m, int nimg, int nz, int nx, int c0, float in_scale, float in_shift,
           const float *__restrict__ v, const float *__restrict__ G,
           __nv_bfloat16 *__restrict__ X)
{
    const size_t total = (size_t)nimg * nx * m * c0;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int c = (int)(e % c0);
        size_t q = e / c0;
        const int col = (int)(q % m);
        q /= m;
        const int x = (int)(q % nx);
        const int img = (int)(q / nx);
        const int b = img * m + col;
        float val = 0.f;
        if (b < nmod)
            val = c < nz ? fmaf(in_scale, v[((size_t)b * nz + c) * nx + x], in_shift)
                         : G[(size_t)x * c0 + c];
        X[e] = __float2bfloat16_rn(val);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_unpack(int nmod, int m, int nz, int nx, int c0, float in_scale,
             const float *__restrict__ dX, float *__restrict__ dv)
{
    const size_t total = (size_t)nmod * nz * nx;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int x = (int)(e % nx);
        const size_t q = e / nx;
        const int z = (int)(q % nz);
        const int b = (int)(q / nz);
        const int img = b / m, col = b - (b / m) * m;
        dv[e] = in_scale * dX[(((size_t)img * nx + x) * m + col) * c0 + z];
    }
}

__global__ void __launch_bounds__(kThreads)
    k_traces(int nmod, int m, int ns, int nr, int nt, int nx, int cout, float amp,
             const int *__restrict__ rec_ix, const float *__restrict__ Y, float *__restrict__ d)
{
    const size_t total = (size_t)nmod * ns * nr * nt;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int t = (int)(e % nt);
        size_t q = e / nt;
        const int r = (int)(q % nr);
        q /= nr;
        const int s = (int)(q % ns);
        const int b = (int)(q / ns);
        const int img = b / m, col = b - (b / m) * m;
        const float y = Y[(((size_t)img * nx + rec_ix[r]) * m + col) * cout + (size_t)s * nt + t];
        d[e] = copysignf(amp * expm1f(fabsf(y)), y);
    }
}

// one thread per output entry of dY (every entry written)
__global__ void __launch_bounds__(kThreads)
    k_outgrad(int nmod, int m, int nimg, int ns, int nr, int nt, int nx, int cout, float amp,
              float scale, const int *__restrict__ col_rec, const float *__restrict__ Y,
              const float *__restrict__ adj, __nv_bfloat16 *__restrict__ dY)
{
    const size_t total = (size_t)nimg * nx * m * cout;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int c = (int)(e % cout);
        size_t q = e / cout;
        const int col = (int)(q % m);
        q /= m;
        const int x = (int)(q % nx);
        const int img = (int)(q / nx);
        const int b = img * m + col, r = col_rec[x];
        float g = 0.f;
        if (b < nmod && r >= 0 && c < ns * nt) {
            const int s = c / nt, t = c - (c / nt) * nt;
            const float a = adj[(((size_t)b * ns + s) * nr + r) * nt + t];
            g = scale * a * amp * expf(fabsf(Y[e]));
        }
        dY[e] = __float2bfloat16_rn(g);
    }
}

__global__ void __launch_bounds__(kThreads)
    k_target(int nmod, int m, int nimg, int ns, int nr, int nt, int nx, int cout, float amp,
             const int *__restrict__ col_rec, const float *__restrict__ d, float *__restrict__ Yt)
{
    const size_t total = (size_t)nimg * nx * m * cout;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int c = (int)(e % cout);
        size_t q = e / cout;
        const int col = (int)(q % m);
        q /= m;
        const int x = (int)(q % nx);
        const int img = (int)(q / nx);
        const int b = img * m + col, r = col_rec[x];
        float y = 0.f;
        if (b < nmod && r >= 0 && c < ns * nt) {
            const int s = c / nt, t = c - (c / nt) * nt;
            const float v = d[(((size_t)b * ns + s) * nr + r) * nt + t];
            y = copysignf(log1pf(fabsf(v) / amp), v);
        }
        Yt[e] = y;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_loss(size_t n, const float *__restrict__ Y, const float *__restrict__ Yt,
           float *__restrict__ part, __nv_bfloat16 *__restrict__ dY)
{
    __shared__ float red[kThreads];
    const float inv = 1.f / (float)n;
    float acc = 0.f;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const float d = Y[e] - Yt[e];
        acc = fmaf(d, d, acc);
        dY[e] = __float2bfloat16_rn(2.f * d * inv);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads)
    k_loss_final(int parts, size_t n, const float *__restrict__ part, float *__restrict__ loss)
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

// row pairs of an image [n][h][w][C] (bf16), 8 channels a thread
__global__ void __launch_bounds__(kThreads)
    k_pool_h(int n, int h, int w, int C, int mode, const uint4 *__restrict__ x,
             uint4 *__restrict__ y)
{
    const int hc = (h + 1) / 2, cg = C / 8;
    const size_t total = (size_t)n * hc * w * cg;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int g = (int)(e % cg);
        size_t q = e / cg;
        const int j = (int)(q % w);
        q /= w;
        const int I = (int)(q % hc);
        const int b = (int)(q / hc);
        const int rows = min(2, h - 2 * I);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < rows; ++k) {
            const uint4 u = x[(((size_t)b * h + 2 * I + k) * w + j) * cg + g];
            const __nv_bfloat162 *hh = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(hh[i]);
                acc[2 * i] += f.x;
                acc[2 * i + 1] += f.y;
            }
        }
        const float s = mode == 0 ? 1.f / (float)rows : 1.f;
        uint4 o;
        __nv_bfloat162 *oh = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
        for (int i = 0; i < 4; ++i) oh[i] = __floats2bfloat162_rn(s * acc[2 * i], s * acc[2 * i + 1]);
        y[e] = o;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_up_h(int n, int ho, int w, int C, int mode, const uint4 *__restrict__ x,
           uint4 *__restrict__ y)
{
    const int hc = (ho + 1) / 2, cg = C / 8;
    const size_t total = (size_t)n * ho * w * cg;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int g = (int)(e % cg);
        size_t q = e / cg;
        const int j = (int)(q % w);
        q /= w;
        const int i = (int)(q % ho);
        const int b = (int)(q / ho);
        const uint4 u = x[(((size_t)b * hc + i / 2) * w + j) * cg + g];
        if (mode == 0) {
            y[e] = u;
        } else {
            const int rows = min(2 * (i / 2) + 2, ho) - 2 * (i / 2);
            const float s = 1.f / (float)rows;
            const __nv_bfloat162 *hh = reinterpret_cast<const __nv_bfloat162 *>(&u);
            uint4 o;
            __nv_bfloat162 *oh = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(hh[k]);
                oh[k] = __floats2bfloat162_rn(s * f.x, s * f.y);
            }
            y[e] = o;
        }
    }
}

__global__ void __launch_bounds__(kThreads)
    k_wprep3(int cout, int cin, const float *__restrict__ W3, __nv_bfloat16 *__restrict__ W,
             __nv_bfloat16 *__restrict__ WT)
{
    const size_t total = (size_t)cout * 9 * cin;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        // W[co][ky][kx][ci]
        const int ci = (int)(e % cin);
        size_t q = e / cin;
        const int kx = (int)(q % 3);
        q /= 3;
        const int ky = (int)(q % 3);
        const int co = (int)(q / 3);
        const float wv = kx == 1 ? W3[((size_t)co * 3 + ky) * cin + ci] : 0.f;
        const __nv_bfloat16 wb = __float2bfloat16_rn(wv);
        W[e] = wb;
        // W^T[ci][2-ky][2-kx][co] = W[co][ky][kx][ci]
        WT[(((size_t)ci * 3 + (2 - ky)) * 3 + (2 - kx)) * cout + co] = wb;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_wcentre(int cout, int cin, const float *__restrict__ dW, float *__restrict__ dW3)
{
    const size_t total = (size_t)cout * 3 * cin;
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < total;
         e += (size_t)gridDim.x * kThreads) {
        const int ci = (int)(e % cin);
        const size_t q = e / cin;     // co * 3 + ky
        dW3[e] = dW[(q * 3 + 1) * cin + ci];
    }
}

__global__ void __launch_bounds__(kThreads)
    k_rel_err(size_t n, const float *__restrict__ g, const float *__restrict__ r,
              float *__restrict__ err)
{
    __shared__ double rn[kThreads], rd[kThreads];
    const size_t off = (size_t)blockIdx.x * n;
    double num = 0.0, den = 0.0;
    for (size_t i = threadIdx.x; i < n; i += kThreads) {
        const double ri = (double)r[off + i];
        const double d = (double)g[off + i] - ri;
        num += d * d;
        den += ri * ri;
    }
    rn[threadIdx.x] = num;
    rd[threadIdx.x] = den;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            rn[threadIdx.x] += rn[threadIdx.x + s];
            rd[threadIdx.x] += rd[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double a = rn[0], b = rd[0];
        err[blockIdx.x] = b > 0.0 ? (float)sqrt(a / b) : (a > 0.0 ? INFINITY : 0.f);
    }
}

fwi_status launch_check(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return FWI_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

fwi_status fwi_sur_pack(int nmod, int m, int nz, int nx, int c0, float in_scale, float in_shift,
                        const float *v, const float *G, void *X, void *stream)
{
    if (nmod < 1 || m < 1 || nz < 1 || nx < 1 || c0 < nz || c0 % 64 != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "nmod, m, nz, nx >= 1 and c0 >= nz a multiple of 64 needed");
    if (!v || !G || !X) return fwi::record_error(FWI_ERR_INVALID_ARG, "v, G and X must not be NULL");
    const int nimg = (nmod + m - 1) / m;
    const size_t n = (size_t)nimg * nx * m * c0;
    k_pack<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(
        nmod, m, nimg, nz, nx, c0, in_scale, in_shift, v, G, static_cast<__nv_bfloat16 *>(X));
    return launch_check("fwi_sur_pack");
}

fwi_status fwi_sur_unpack_grad(int nmod, int m, int nz, int nx, int c0, float in_scale,
                               const float *dX, float *dv, void *stream)
{
    if (nmod < 1 || m < 1 || nz < 1 || nx < 1 || c0 < nz)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "nmod, m, nz, nx >= 1 and c0 >= nz needed");
    if (!dX || !dv) return fwi::record_error(FWI_ERR_INVALID_ARG, "dX and dv must not be NULL");
    const size_t n = (size_t)nmod * nz * nx;
    k_unpack<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(nmod, m, nz, nx, c0, in_scale,
                                                                  dX, dv);
    return launch_check("fwi_sur_unpack_grad");
}

fwi_status fwi_sur_traces(int nmod, int m, int ns, int nr, int nt, int nx, int cout, float amp,
                          const int *rec_ix, const float *Y, float *d, void *stream)
{
    if (nmod < 1 || m < 1 || ns < 1 || nr < 1 || nt < 1 || nx < 1 || (long long)ns * nt > cout ||
        !(amp > 0.f))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "sizes >= 1, ns nt <= cout and amp > 0 needed");
    if (!rec_ix || !Y || !d)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "rec_ix, Y and d must not be NULL");
    const size_t n = (size_t)nmod * ns * nr * nt;
    k_traces<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(nmod, m, ns, nr, nt, nx, cout,
                                                                  amp, rec_ix, Y, d);
    return launch_check("fwi_sur_traces");
}

fwi_status fwi_sur_output_grad(int nmod, int m, int ns, int nr, int nt, int nx, int cout,
                               float amp, float scale, const int *col_rec, const float *Y,
                               const float *adj, void *dY, void *stream)
{
    if (nmod < 1 || m < 1 || ns < 1 || nr < 1 || nt < 1 || nx < 1 || (long long)ns * nt > cout ||
        !(amp > 0.f))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "sizes >= 1, ns nt <= cout and amp > 0 needed");
    if (!col_rec || !Y || !adj || !dY)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "col_rec, Y, adj and dY must not be NULL");
    const int nimg = (nmod + m - 1) / m;
    const size_t n = (size_t)nimg * nx * m * cout;
    k_outgrad<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(
        nmod, m, nimg, ns, nr, nt, nx, cout, amp, scale, col_rec, Y, adj,
        static_cast<__nv_bfloat16 *>(dY));
    return launch_check("fwi_sur_output_grad");
}

fwi_status fwi_sur_target(int nmod, int m, int ns, int nr, int nt, int nx, int cout, float amp,
                          const int *col_rec, const float *d, float *Yt, void *stream)
{
    if (nmod < 1 || m < 1 || ns < 1 || nr < 1 || nt < 1 || nx < 1 || (long long)ns * nt > cout ||
        !(amp > 0.f))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "sizes >= 1, ns nt <= cout and amp > 0 needed");
    if (!col_rec || !d || !Yt)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "col_rec, d and Yt must not be NULL");
    const int nimg = (nmod + m - 1) / m;
    const size_t n = (size_t)nimg * nx * m * cout;
    k_target<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(nmod, m, nimg, ns, nr, nt, nx,
                                                                  cout, amp, col_rec, d, Yt);
    return launch_check("fwi_sur_target");
}

fwi_status fwi_sur_loss(long long n, const float *Y, const float *Yt, float *loss, void *dY,
                        float *work, long long work_floats, void *stream)
{
    if (n < 1) return fwi::record_error(FWI_ERR_INVALID_ARG, "n must be >= 1");
    if (!Y || !Yt || !loss || !dY || !work || work_floats < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "Y, Yt, loss, dY and a work buffer are needed");
    const long long g = work_floats < kLossCtas ? work_floats : kLossCtas;
    cudaStream_t st = (cudaStream_t)stream;
    k_loss<<<(unsigned)g, kThreads, 0, st>>>((size_t)n, Y, Yt, work,
                                             static_cast<__nv_bfloat16 *>(dY));
    k_loss_final<<<1, kThreads, 0, st>>>((int)g, (size_t)n, work, loss);
    return launch_check("fwi_sur_loss");
}

fwi_status fwi_pool_h_bf16(int n, int h, int w, int channels, int mode, const void *x, void *y,
                           void *stream)
{
    if (n < 1 || h < 1 || w < 1 || channels < 8 || channels % 8 != 0 || (mode != 0 && mode != 1))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "n, h, w >= 1, channels a multiple of 8, mode 0 or 1 needed");
    if (!x || !y || !aligned16(x) || !aligned16(y))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    const size_t e = (size_t)n * ((h + 1) / 2) * w * (channels / 8);
    k_pool_h<<<grid_for(e), kThreads, 0, (cudaStream_t)stream>>>(
        n, h, w, channels, mode, static_cast<const uint4 *>(x), static_cast<uint4 *>(y));
    return launch_check("fwi_pool_h_bf16");
}

fwi_status fwi_up_h_bf16(int n, int ho, int w, int channels, int mode, const void *x, void *y,
                         void *stream)
{
    if (n < 1 || ho < 1 || w < 1 || channels < 8 || channels % 8 != 0 || (mode != 0 && mode != 1))
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "n, ho, w >= 1, channels a multiple of 8, mode 0 or 1 needed");
    if (!x || !y || !aligned16(x) || !aligned16(y))
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    const size_t e = (size_t)n * ho * w * (channels / 8);
    k_up_h<<<grid_for(e), kThreads, 0, (cudaStream_t)stream>>>(
        n, ho, w, channels, mode, static_cast<const uint4 *>(x), static_cast<uint4 *>(y));
    return launch_check("fwi_up_h_bf16");
}

fwi_status fwi_sur_weights_prep(int cout, int cin, const float *W3, void *W, void *WT,
                                void *stream)
{
    if (cout < 1 || cin < 1) return fwi::record_error(FWI_ERR_INVALID_ARG, "cout, cin >= 1");
    if (!W3 || !W || !WT)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "W3, W and WT must not be NULL");
    const size_t n = (size_t)cout * 9 * cin;
    k_wprep3<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(
        cout, cin, W3, static_cast<__nv_bfloat16 *>(W), static_cast<__nv_bfloat16 *>(WT));
    return launch_check("fwi_sur_weights_prep");
}

fwi_status fwi_sur_wgrad_centre(int cout, int cin, const float *dW, float *dW3, void *stream)
{
    if (cout < 1 || cin < 1) return fwi::record_error(FWI_ERR_INVALID_ARG, "cout, cin >= 1");
    if (!dW || !dW3) return fwi::record_error(FWI_ERR_INVALID_ARG, "dW and dW3 must not be NULL");
    const size_t n = (size_t)cout * 3 * cin;
    k_wcentre<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(cout, cin, dW, dW3);
    return launch_check("fwi_sur_wgrad_centre");
}

fwi_status fwi_rel_error(int nmod, long long n, const float *g, const float *g_ref, float *err,
                         void *stream)
{
    if (nmod < 1 || n < 1) return fwi::record_error(FWI_ERR_INVALID_ARG, "nmod, n >= 1");
    if (!g || !g_ref || !err)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "g, g_ref and err must not be NULL");
    k_rel_err<<<(unsigned)nmod, kThreads, 0, (cudaStream_t)stream>>>((size_t)n, g, g_ref, err);
    return launch_check("fwi_rel_error");
}

}  // extern "C"
