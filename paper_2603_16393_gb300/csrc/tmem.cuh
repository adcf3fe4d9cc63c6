// tmem.cuh -- tensor memory as per-thread storage for the propagators, and
// the L2 bulk prefetch of their record planes.
//
// A CTA allocates `cols` columns (a power of two, 32..512) once; thread t of
// warp w reads and writes its own lane 32 (w mod 4) + (t mod 32) with the
// 32x32b shapes, so each warp of a lane quarter takes its own range of
// columns.  The loads and stores are warp-collective (.sync.aligned): every
// thread of a warp executes them, inactive threads on harmless columns.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fwi {
namespace {

// warp 0 allocates (and gives up the permit to allocate again: one
// allocation per CTA); the address comes back through shared memory
__device__ __forceinline__ uint32_t tmem_alloc(uint32_t *slot, uint32_t cols)
{
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *slot;
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(cols)
                     : "memory");
    }
}

// L2 prefetch of a record plane (16-byte aligned, size a multiple of 16) in
// 4 KB pieces, one piece per thread of the first warps
__device__ __forceinline__ void prefetch_plane_l2(const float *p, size_t bytes, int tid)
{
    const size_t off = (size_t)tid * 4096;
    if (off < bytes) {
        const unsigned n = (unsigned)min((size_t)4096, bytes - off);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char *)p + off),
                     "r"(n)
                     : "memory");
    }
}

// two fp32 columns of this thread's TMEM lane (warp-collective; the values
// are valid after tmem_wait_ld)
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t &a, uint32_t &b)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(a), "=r"(b)
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t &a, uint32_t &b, uint32_t &c,
                                         uint32_t &d)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float2 u, float2 v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(u.x)), "r"(__float_as_uint(u.y)), "r"(__float_as_uint(v.x)),
                 "r"(__float_as_uint(v.y))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st2(uint32_t taddr, float2 v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace
}  // namespace fwi
