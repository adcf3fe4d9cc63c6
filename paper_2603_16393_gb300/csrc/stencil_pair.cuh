// stencil_pair.cuh -- one time step of a thread's column pair in the
// on-chip propagators (resident and cluster kernels): the thread owns columns
// (x, x+1) and RW consecutive rows of a field held in shared memory at row
// pitch P (two ghost rows and columns around), moves them as 8-byte accesses
// and updates both cells with the packed f32x2 instructions (results bitwise
// those of the scalar operations on each cell).
//
// fwd_rows_pair: increment form of the damped leapfrog of Eq. 1,
//   v^{j+1/2} = AB v^{j-1/2} + kappa A (L u^j),  u^{j+1} = u^j + v^{j+1/2},
//   the 4th-order Laplacian on neighbour differences; kappa A and v of the
//   RW x 2 cells in registers, A B from a shared table (abp, pitch P); the
//   record plane gets L u^j (sw, pitch PR).
// adj_rows_pair: the same propagator on reversed time in the phi = kappa A mu
//   form, phi^{j-1} = kappa A (L^T phi^j) + 2A phi^j - AB phi^{j+1}; the
//   imaging sums and (kappa A, 2A) of the cells in the thread's TMEM lane
//   (tacc: 2 columns a row; tkd: 4 columns a row), the record read through a
//   ring of KR rows in flight (rq), imaging acc += phi^{j-1} t.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "f32x2.cuh"
#include "fwi_internal.cuh"
#include "tmem.cuh"

namespace fwi {
namespace {

template <int P, int PR, int RW, int TOPBC, bool STORE, bool AHEAD>
__device__ __forceinline__ void fwd_rows_pair(const float *__restrict__ cp, float *__restrict__ np,
                                              const float *__restrict__ abp,
                                              float *__restrict__ sw, bool top_strip,
                                              const float2 (&ka)[RW], float2 (&vi)[RW],
                                              const PropArgs &a)
{
    using namespace f2;
    const float2 CX1 = splat(a.cx1), CX2 = splat(a.cx2), CZ1 = splat(a.cz1), CZ2 = splat(a.cz2);
    float2 wm2 = ld(cp - 2 * P), wm1 = ld(cp - P), w0 = ld(cp), wp1 = ld(cp + P);
    // AHEAD: the shared-memory operands of row r + 1 are loaded while row r
    // is updated (a row's arithmetic is a chain of dependent packed
    // operations); the queue kernel, whose plan-indexed arguments hold more
    // registers, loads each row's operands in its own iteration
    float2 nwp2 = {}, nL = {}, nR = {}, nab = {};
    if (AHEAD) nwp2 = ld(cp + 2 * P), nL = ld(cp - 2), nR = ld(cp + 2), nab = ld(abp);
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const float *c = cp + r * P;
        const float2 wp2 = AHEAD ? nwp2 : ld(c + 2 * P);
        const float2 L = AHEAD ? nL : ld(c - 2);     // u[x-2], u[x-1]
        const float2 R = AHEAD ? nR : ld(c + 2);     // u[x+2], u[x+3]
        const float2 ab_ahead = nab;
        if (AHEAD && r + 1 < RW) {
            nwp2 = ld(c + 3 * P);
            nL = ld(c + P - 2);
            nR = ld(c + P + 2);
            nab = ld(abp + (r + 1) * P);
        }
        // x, first neighbours: (u[x-1] - u[x]) + (u[x+1] - u[x]) per column
        const float d01 = w0.y - w0.x;
        const float2 dxA = make_float2((L.y - w0.x) + d01, (R.x - w0.y) - d01);
        // x, second neighbours; z
        const float2 dxB = add(sub(L, w0), sub(R, w0));
        const float2 dzA = add(sub(wm1, w0), sub(wp1, w0));
        const float2 dzB = add(sub(wm2, w0), sub(wp2, w0));
        float2 lap = mul(CX1, dxA);
        lap = fma(CX2, dxB, lap);
        lap = fma(CZ1, dzA, lap);
        lap = fma(CZ2, dzB, lap);
        const float2 ab = AHEAD ? ab_ahead : ld(abp + r * P);
        vi[r] = fma(ka[r], lap, mul(ab, vi[r]));
        const float2 un = add(w0, vi[r]);
        st(np + r * P, un);
        if (TOPBC == 1 && (r == 1 || r == 2)) {
            if (top_strip) st(np - r * P, un);   // mirrored ghost rows -1, -2
        }
        if (STORE) st(sw + r * PR, lap);
        wm2 = wm1;
        wm1 = w0;
        w0 = wp1;
        wp1 = wp2;
    }
}

template <int P, int PR, int RW, int KR, int TOPBC>
__device__ __forceinline__ void adj_rows_pair(const float *__restrict__ cp,
                                              float *__restrict__ np,
                                              const float *__restrict__ sr,
                                              const float *__restrict__ sr_next,
                                              bool top_strip, bool active, uint32_t tacc,
                                              uint32_t tkd, float2 (&rq)[KR], const PropArgs &a)
{
    using namespace f2;
    const float2 &C0 = a.w2[0], &CX1 = a.w2[1], &CX2 = a.w2[2], &CZ1 = a.w2[3], &CZ2 = a.w2[4];
    float2 wm2 = ld(cp - 2 * P), wm1 = ld(cp - P), w0 = ld(cp), wp1 = ld(cp + P);
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const float *c = cp + r * P;
        const float2 wp2 = ld(c + 2 * P);
        const float2 L = ld(c - 2);     // u[x-2], u[x-1]
        const float2 R = ld(c + 2);     // u[x+2], u[x+3]
        float2 lap = mul(C0, w0);
        lap = fma(CX1, make_float2(L.y + w0.y, w0.x + R.x), lap);
        lap = fma(CX2, add(L, R), lap);
        lap = fma(CZ1, add(wm1, wp1), lap);
        lap = fma(CZ2, add(wm2, wp2), lap);
        if (TOPBC == 1 && (r == 1 || r == 2)) {
            // transpose of the mirrored top: reflected weights back onto rows 1, 2
            if (top_strip) lap = (r == 1) ? add(lap, fma(CZ2, w0, mul(CZ1, wm1)))
                                          : fma(CZ2, wm2, lap);
        }
        uint32_t s0, s1, k0, k1, d0, d1;
        tmem_ld2(tacc + 2 * r, s0, s1);
        tmem_ld4(tkd + 4 * r, k0, k1, d0, d1);
        const float2 fo = ld(np + r * P);
        tmem_wait_ld();
        const float2 kA = make_float2(__uint_as_float(k0), __uint_as_float(k1));
        const float2 A2 = make_float2(__uint_as_float(d0), __uint_as_float(d1));   // 2A
        const float2 nAB = fma(A2, splat(-1.f), splat(1.f));            // -A B = 1 - 2A
        const float2 fn = fma(kA, lap, fma(A2, w0, mul(nAB, fo)));
        if (active) st(np + r * P, fn);
        tmem_st2(tacc + 2 * r,
                 fma(fn, rq[0], make_float2(__uint_as_float(s0), __uint_as_float(s1))));
#pragma unroll
        for (int i = 0; i + 1 < KR; ++i) rq[i] = rq[i + 1];
        rq[KR - 1] = (r + KR < RW) ? ld(sr + (r + KR) * PR) : ld(sr_next + (r + KR - RW) * PR);
        wm2 = wm1;
        wm1 = w0;
        w0 = wp1;
        wp1 = wp2;
    }
}

}  // namespace
}  // namespace fwi
