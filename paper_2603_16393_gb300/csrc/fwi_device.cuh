// fwi_device.cuh -- device helpers shared by the propagators: the Ricker
// source and the damping / per-cell coefficients of Eq. 1 with the absorbing
// layer (Sec. 6.1).  Templates on the kernel argument block, which provides
// nz, nx, nb, dtd, t0d, fp, src_scale, ex0, ez0, ex0d, ez0d, inv_nb.
#pragma once

#include <cuda_runtime.h>

namespace fwi {
namespace dev {

constexpr float kPi = 3.14159265358979323846f;

// Ricker wavelet at t = j dt - t0 (time formed in double), times 1/(dx dz)
template <class A>
__device__ __forceinline__ float ricker_scaled(int j, const A &a)
{
    const float t = (float)((double)j * a.dtd - a.t0d);
    const float q = (kPi * a.fp * t) * (kPi * a.fp * t);
    return a.src_scale * (1.f - 2.f * q) * expf(-q);
}

// damping e = eta dt / 2 of column x (side layers)
template <class A>
__device__ __forceinline__ float ex_of(int x, const A &a)
{
    float cxd = 0.f;
    if (x < a.nb) cxd = (float)(a.nb - x);
    else if (x > a.nb + a.nx - 1) cxd = (float)(x - (a.nb + a.nx - 1));
    return a.ex0 * (cxd * a.inv_nb) * (cxd * a.inv_nb);
}

// damping e of row z (bottom layer), as a function of z - (nz - 1): exact
// small integers in float
template <class A>
__device__ __forceinline__ float ez_of(float zbr, const A &a)
{
    const float cz = fmaxf(zbr, 0.f) * a.inv_nb;
    return a.ez0 * cz * cz;
}

// Per-cell coefficients formed in double and rounded once (set-up only):
// kappa A = (v dt)^2 / (1 + e), A B = (1 - e) / (1 + e), kappa / B.  Forming
// (v dt)^2 from a float dt would bias every cell's velocity by the same
// ~5e-8 and shift all arrivals coherently over a thousand steps.
template <class A>
__device__ __forceinline__ double e_cell(int px, int pz, const A &a)
{
    double cx = 0.0, cz = 0.0;
    if (px < a.nb) cx = a.nb - px;
    else if (px > a.nb + a.nx - 1) cx = px - (a.nb + a.nx - 1);
    if (pz > a.nz - 1) cz = pz - (a.nz - 1);
    if (a.nb == 0) return 0.0;
    return a.ex0d * (cx / a.nb) * (cx / a.nb) + a.ez0d * (cz / a.nb) * (cz / a.nb);
}

template <class A>
__device__ __forceinline__ float kappaA_cell(float v, int px, int pz, const A &a)
{
    const double vdt = (double)v * a.dtd;
    return (float)(vdt * vdt / (1.0 + e_cell(px, pz, a)));
}

}  // namespace dev
}  // namespace fwi
