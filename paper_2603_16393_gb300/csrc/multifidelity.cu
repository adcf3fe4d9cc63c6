// multifidelity.cu -- the grid transfers of the low-fidelity guidance
// surrogate (the multi-fidelity route to cheaper physics guidance, Sec. 7):
// the W2 potential of a problem coarsened by two in space and time is
// evaluated at R v, and its gradient returns to the fine grid through R^T.
//   k_restrict2:   vc[b][I][J] = mean of v[b][2I..2I+1][2J..2J+1] inside the grid
//   k_restrict2_t: g[b][i][j]  = gc[b][i/2][j/2] / (cells averaged into it)
//   k_decimate2:   dc[b][s][r][m] = d[b][s][2r][2m+1], m < nt/2 (fine sample
//                  n holds t = (n+1) dt, coarse sample m holds t = (m+1) 2 dt)
// One thread per output element, grid-stride.
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

__global__ void __launch_bounds__(kThreads)
    k_restrict2(size_t n, int nz, int nx, int nzc, int nxc, const float *__restrict__ v,
                float *__restrict__ vc)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const size_t b = e / ((size_t)nzc * nxc);
        const int r = (int)(e - b * (size_t)nzc * nxc);
        const int I = r / nxc, J = r - (r / nxc) * nxc;
        const float *vb = v + b * (size_t)nz * nx;
        const int i0 = 2 * I, j0 = 2 * J;
        const int i1 = min(i0 + 2, nz), j1 = min(j0 + 2, nx);
        float s = 0.f;
        for (int i = i0; i < i1; ++i)
            for (int j = j0; j < j1; ++j) s += vb[(size_t)i * nx + j];
        vc[e] = s / (float)((i1 - i0) * (j1 - j0));
    }
}

__global__ void __launch_bounds__(kThreads)
    k_restrict2_t(size_t n, int nz, int nx, int nzc, int nxc, const float *__restrict__ gc,
                  float *__restrict__ g)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const size_t b = e / ((size_t)nz * nx);
        const int r = (int)(e - b * (size_t)nz * nx);
        const int i = r / nx, j = r - (r / nx) * nx;
        const int I = i / 2, J = j / 2;
        const int cnt = (min(2 * I + 2, nz) - 2 * I) * (min(2 * J + 2, nx) - 2 * J);
        g[e] = gc[b * (size_t)nzc * nxc + (size_t)I * nxc + J] / (float)cnt;
    }
}

__global__ void __launch_bounds__(kThreads)
    k_decimate2(size_t n, int nr, int nt, int nrc, int ntc, const float *__restrict__ d,
                float *__restrict__ dc)
{
    for (size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x; e < n;
         e += (size_t)gridDim.x * kThreads) {
        const size_t tr = e / ntc;                  // (b, s, rc) flattened
        const int m = (int)(e - tr * ntc);
        const size_t bs = tr / nrc;
        const int rc = (int)(tr - bs * nrc);
        dc[e] = d[(bs * nr + 2 * (size_t)rc) * nt + 2 * (size_t)m + 1];
    }
}

fwi_status launch_check(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_restrict2(int batch, int nz, int nx, const float *v, float *vc, void *stream)
{
    if (batch < 1 || nz < 1 || nx < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "batch, nz, nx must be >= 1");
    if (!v || !vc) return fwi::record_error(FWI_ERR_INVALID_ARG, "v and vc must not be NULL");
    const int nzc = (nz + 1) / 2, nxc = (nx + 1) / 2;
    const size_t n = (size_t)batch * nzc * nxc;
    k_restrict2<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(n, nz, nx, nzc, nxc, v, vc);
    return launch_check("fwi_restrict2");
}

fwi_status fwi_restrict2_transpose(int batch, int nz, int nx, const float *gc, float *g,
                                   void *stream)
{
    if (batch < 1 || nz < 1 || nx < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "batch, nz, nx must be >= 1");
    if (!gc || !g) return fwi::record_error(FWI_ERR_INVALID_ARG, "gc and g must not be NULL");
    const int nzc = (nz + 1) / 2, nxc = (nx + 1) / 2;
    const size_t n = (size_t)batch * nz * nx;
    k_restrict2_t<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(n, nz, nx, nzc, nxc, gc, g);
    return launch_check("fwi_restrict2_transpose");
}

fwi_status fwi_decimate2(int batch, int ns, int nr, int nt, const float *d, float *dc,
                         void *stream)
{
    if (batch < 1 || ns < 1 || nr < 1 || nt < 2)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "batch, ns, nr >= 1 and nt >= 2 needed");
    if (!d || !dc) return fwi::record_error(FWI_ERR_INVALID_ARG, "d and dc must not be NULL");
    const int nrc = (nr + 1) / 2, ntc = nt / 2;
    const size_t n = (size_t)batch * ns * nrc * ntc;
    k_decimate2<<<grid_for(n), kThreads, 0, (cudaStream_t)stream>>>(n, nr, nt, nrc, ntc, d, dc);
    return launch_check("fwi_decimate2");
}

fwi_status fwi_coarse_problem(const fwi_problem *fine, fwi_problem *coarse, int *src_iz,
                              int *src_ix, int *rec_iz, int *rec_ix)
{
    if (!fine || !coarse || !src_iz || !src_ix || !rec_iz || !rec_ix)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "fine, coarse and the four index arrays must not be NULL");
    if (!fine->src_iz || !fine->src_ix || !fine->rec_iz || !fine->rec_ix)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "the fine problem's index arrays are NULL");
    if (fine->nz < 1 || fine->nx < 1 || fine->nb < 0 || fine->ns < 1 || fine->nr < 1 ||
        fine->ns > FWI_MAX_SHOTS || fine->nr > FWI_MAX_RECEIVERS)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "fine grid, layer, shot or receiver counts out of range");
    if (fine->nt < 4)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "nt = %d: the coarse problem needs nt / 2 >= 2 steps", fine->nt);
    fwi_problem c = *fine;
    c.nz = (fine->nz + 1) / 2;
    c.nx = (fine->nx + 1) / 2;
    c.nb = (fine->nb + 1) / 2;
    c.nt = fine->nt / 2;
    c.dz = 2.0 * fine->dz;
    c.dx = 2.0 * fine->dx;
    c.dt = 2.0 * fine->dt;
    c.checkpoint_every = fine->checkpoint_every ? (fine->checkpoint_every + 1) / 2 : 0;
    for (int i = 0; i < fine->ns; ++i) {
        src_iz[i] = fine->src_iz[i] / 2;
        src_ix[i] = fine->src_ix[i] / 2;
    }
    int nrc = 0;
    for (int i = 0; i < fine->nr; i += 2, ++nrc) {   // the even receivers
        rec_iz[nrc] = fine->rec_iz[i] / 2;
        rec_ix[nrc] = fine->rec_ix[i] / 2;
    }
    c.nr = nrc;
    c.src_iz = src_iz;
    c.src_ix = src_ix;
    c.rec_iz = rec_iz;
    c.rec_ix = rec_ix;
    *coarse = c;
    return FWI_OK;
}

}  // extern "C"
