// conv_tc.cu -- 3x3 convolution (stride 1, zero padding 1) on the fifth-
// generation tensor cores, the dense contraction of a convolutional score or
// surrogate network for the guidance of Algorithms 1-2:
//
//   y[n][p][co] = act(bias[co] + sum_{tap, ci} x[n][p + tap][ci] w[co][tap][ci])
//
// as an implicit GEMM: M = 128 output pixels (an 8 x 16 tile of one image),
// N = 256 output channels (cout a multiple of 256), K = 9 taps x cin.
// Layouts: x NHWC bf16, w [cout][3][3][cin] bf16 (K-major), y NHWC fp32 or
// bf16.  The MMA rate per SM grows with N: 1.50 PFLOP/s at N = 256 (a 256 ->
// 256 layer), 0.76 at N = 128 (128 -> 128), 152 x 70 x 70; every other cout
// therefore runs k_conv3x3_tc_pn below in 128-channel blocks (a 64-channel
// remainder on zero-filled weight rows), pixels as N = 192
// (1.03 PFLOP/s on the 128 -> 128 layer).
//
// Operand A comes from one halo box per 64-channel block: the 10 x 18 pixels
// around the tile (a 4D cp.async.bulk.tensor load, 128-byte swizzled, one
// 128-byte row per pixel; pixels outside the image read the zero fill, which
// is the padding).  The nine tap-shifted 128 x 64 operands are views into it:
// view (dy, dx) starts at halo row 10 (dy + 1) + dx + 1 and its 8-row groups
// (one image row of the tile each) are 10 rows = 1280 bytes apart; the
// swizzle follows the absolute address, so neither the unaligned start rows
// nor the 1280-byte group stride needs a base offset.  A is thus read once
// per channel block instead of nine times.
// Operand B, the weight block of one tap and channel block, streams through
// its own ring.
//
// A persistent kernel, one CTA of eighteen warps per SM, tiles handed out
// round-robin:
//   * warp 0 (one thread) is the TMA producer, loading halo boxes and weight
//     blocks in the order the MMAs consume them;
//   * warp 1 allocates the tensor memory, and one of its threads issues the
//     tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators of 128 lanes x
//     BN columns) into one of two accumulators, returning ring stages and
//     handing finished accumulators on through tcgen05.commit;
//   * warps 2-17 are the epilogue: they read an accumulator back (tcgen05.ld;
//     warp w owns lanes 32 (w mod 4) .. +31, i.e. those pixels, and a quarter
//     of the columns), add the bias, apply the activation, store the pixels
//     inside the image and release the accumulator, while the MMAs of the
//     next tile fill the other one.  Sixteen warps, because with four the
//     epilogue (not the MMAs) set the pace: 0.51 against 0.29 ms at 152 x
//     70 x 70 x 128 -> 128.
// Every mbarrier wait is bounded in time; a wait that runs out records
// FWI_ERR_DEVICE_TIMEOUT in the caller's status word, and every role then
// stops (the outputs are incomplete) and the CTA releases its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "fwi_internal.cuh"
#include "silu.cuh"

namespace {

constexpr int kTW = 8, kTH = 16, kBM = kTW * kTH;   // output pixels per tile (the MMA's M)
constexpr int kBK = 64;                              // channels per K block (128 bytes of bf16)
constexpr int kHX = kTW + 2, kHY = kTH + 2;          // halo box: 10 x 18 pixels (x0-1 .. x0+8)
constexpr int kHaloTx = kHX * kHY * kBK * 2;          // bytes one halo load delivers (22.5 KB)
constexpr int kHaloBytes = (kHaloTx + 1023) / 1024 * 1024;   // its 1024-aligned slot (23 KB)
constexpr int kAStages = 2;
// weight-block ring: 8 stages of BN x 64 channels, 5 when BN = 256 (32 KB each)
template <int BN> __host__ __device__ constexpr int b_stages() { return BN == 256 ? 5 : 8; }
constexpr int kThreads = 576;                        // producer, MMA, sixteen epilogue warps
constexpr int kEpiWarps = 16;
constexpr unsigned long long kWaitNs = 2000000000ull;   // bound of one mbarrier wait: 2 s
constexpr unsigned long long kCheckWaitNs = 20000000ull; // the wait self-check: 20 ms

struct ConvArgs {
    unsigned long long wait_ns;    // bound of one mbarrier wait
    int withhold;                  // 1: never load the weight blocks (the wait self-check)
    int n, h, w, cin, cout;
    int act;       // 0: none, 1: SiLU, 2: y = bf16(pre-activation), y2 = bf16(SiLU(y)),
                   // 3: y = bf16(bf16(conv) silu'(y2)) with y2 a bf16 input

    int y_bf16;    // output type: 0 fp32, 1 bf16
    int tiles_x, tiles_y, tiles;   // pixel tiles per image row / column, tiles in all
    const float *bias;
    void *y;
    int *status;
    void *y2;      // act 2: the activation out; act 3: the pre-activation in (bf16, y's layout)
};

__device__ __forceinline__ unsigned su32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mb_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mb_try(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the completion of the barrier phase of the given parity; false
// once *failed is set (failed may be NULL) or after limit_ns (then it sets
// *failed).
__device__ __forceinline__ bool mb_wait(uint64_t *b, unsigned parity, volatile int *failed,
                                        unsigned long long limit_ns)
{
    if (mb_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mb_try(b, parity)) return true;
        if (failed && *failed) return false;
        if (now_ns() - t0 > limit_ns) {
            if (failed) *failed = 1;
            return false;
        }
    }
}

// After a failed wait the producer waits (bounded) for the loads it issued
// into each stage, so that no copy still writes into this CTA's shared memory
// when it exits: stage s last received load number last[s] (-1: none), whose
// full barrier completes phase last[s] / stages.
template <int S>
__device__ __forceinline__ void drain_loads(uint64_t *full, const int (&last)[S],
                                            unsigned long long limit_ns)
{
    for (int s = 0; s < S; ++s)
        if (last[s] >= 0) mb_wait(&full[s], (unsigned)((last[s] / S) & 1), nullptr, limit_ns);
}

__device__ __forceinline__ void mb_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void mb_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_4d(void *dst, const CUtensorMap *m, int c0, int c1, int c2,
                                       int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *m, int c0, int c1,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(c0), "r"(c1), "r"(su32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in a 128-byte-swizzled
// buffer written by TMA: rows of 128 bytes, 8-row groups `group_bytes` apart
// (stride byte offset), descriptor version 1, swizzle mode 128 B, base offset
// 0.  The swizzle pattern follows the absolute shared-memory address (the
// TMA wrote it that way into a 1024-byte-aligned buffer), so a view may start
// at any 128-byte row of the buffer.
__device__ __forceinline__ uint64_t sw128_desc(const void *start, uint32_t group_bytes)
{
    const uint64_t a = su32(start);
    return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(group_bytes >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrives on the mbarrier once every tcgen05.mma issued so far by this
// thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive fp32 columns of this warp's 32 accumulator lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float v) { return __fdividef(v, 1.f + __expf(-v)); }

// Tile t -> image, pixel-tile origin and output-channel block (channel block
// slowest, so the CTAs running at once share the weight blocks)
struct Tile {
    int img, x0, y0, n0;
};
__device__ __forceinline__ Tile tile_of(int t, const ConvArgs &a, int BN)
{
    const int per_block = a.tiles;
    Tile r;
    const int cbk = t / per_block;
    t -= cbk * per_block;
    const int tx = t % a.tiles_x;
    t /= a.tiles_x;
    const int ty = t % a.tiles_y;
    r.img = t / a.tiles_y;
    r.x0 = tx * kTW;
    r.y0 = ty * kTH;
    r.n0 = cbk * BN;
    return r;
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv3x3_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
                 const ConvArgs a)
{
    constexpr int kBBytes = BN * kBK * 2;
    constexpr int kBStages = b_stages<BN>();
    constexpr uint32_t kIdesc = idesc_bf16(BN);
    constexpr uint32_t kTmemCols = 2 * BN;   // two accumulators
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sA = base;                           // kAStages halo boxes
    unsigned char *sB = base + kAStages * kHaloBytes;   // kBStages weight blocks
    __shared__ uint64_t a_full[kAStages], a_empty[kAStages], b_full[kBStages], b_empty[kBStages];
    __shared__ uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    volatile int *vfailed = &failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cbs = a.cin / kBK;
    const int total = a.tiles * (a.cout / BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mb_init(&a_full[s], 1);
            mb_init(&a_empty[s], 1);
        }
        for (int s = 0; s < kBStages; ++s) {
            mb_init(&b_full[s], 1);
            mb_init(&b_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mb_init(&acc_full[b], 1);
            mb_init(&acc_empty[b], kEpiWarps);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer, in the MMAs' order: per tile and channel block the
            // halo box, then the nine weight blocks of that channel block
            int ga = 0, gb = 0;
            int last_a[kAStages], last_b[kBStages];
            for (int s = 0; s < kAStages; ++s) last_a[s] = -1;
            for (int s = 0; s < kBStages; ++s) last_b[s] = -1;
            for (int t = blockIdx.x; t < total && !*vfailed; t += gridDim.x) {
                const Tile tl = tile_of(t, a, BN);
                for (int cb = 0; cb < cbs && !*vfailed; ++cb) {
                    const int sa = ga % kAStages, ra = ga / kAStages;
                    if (ra > 0 && !mb_wait(&a_empty[sa], (unsigned)((ra - 1) & 1), vfailed, a.wait_ns)) break;
                    mb_expect(&a_full[sa], kHaloTx);
                    tma_4d(sA + sa * kHaloBytes, &tmx, cb * kBK, tl.x0 - 1, tl.y0 - 1, tl.img,
                           &a_full[sa]);
                    last_a[sa] = ga++;
                    for (int tap = 0; tap < 9; ++tap, ++gb) {
                        const int sb = gb % kBStages, rb = gb / kBStages;
                        if (rb > 0 && !mb_wait(&b_empty[sb], (unsigned)((rb - 1) & 1), vfailed, a.wait_ns))
                            break;
                        if (a.withhold) continue;
                        mb_expect(&b_full[sb], kBBytes);
                        tma_2d(sB + sb * kBBytes, &tmw, tap * a.cin + cb * kBK, tl.n0, &b_full[sb]);
                        last_b[sb] = gb;
                    }
                }
            }
            if (*vfailed) {
                drain_loads(a_full, last_a, a.wait_ns);
                drain_loads(b_full, last_b, a.wait_ns);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile number it fills accumulator it & 1 once the
            // epilogue has released its previous use; per tap four K = 16
            // steps, advancing the start address by 32 bytes inside the
            // swizzled 128-byte rows
            int ga = 0, gb = 0, it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok && !*vfailed; t += gridDim.x, ++it) {
                const int b = it & 1, u = it >> 1;
                if (u > 0 && !mb_wait(&acc_empty[b], (unsigned)((u - 1) & 1), vfailed, a.wait_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int cb = 0; cb < cbs && ok; ++cb, ++ga) {
                    const int sa = ga % kAStages, ra = ga / kAStages;
                    if (!mb_wait(&a_full[sa], (unsigned)(ra & 1), vfailed, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const unsigned char *halo = sA + sa * kHaloBytes;
                    for (int tap = 0; tap < 9; ++tap, ++gb) {
                        const int sb = gb % kBStages, rb = gb / kBStages;
                        if (!mb_wait(&b_full[sb], (unsigned)(rb & 1), vfailed, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int row = (tap / 3) * kHX + tap % 3;   // (dy + 1) 10 + dx + 1
                        const uint64_t ad = sw128_desc(halo + row * 128, kHX * 128);
                        const uint64_t bd = sw128_desc(sB + sb * kBBytes, 1024);
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k)
                            umma_bf16(d, ad + 2 * k, bd + 2 * k, kIdesc,
                                      (cb | tap | k) != 0);
                        umma_commit(&b_empty[sb]);
                    }
                    if (ok) umma_commit(&a_empty[sa]);
                }
                if (ok) umma_commit(&acc_full[b]);
            }
        }
    } else {
        // epilogue warps 2..17: lanes 32 (warp mod 4) .. +31 of the accumulator
        // (the lane quarter a warp may access), and one quarter of its columns
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int part = (warp - 2) >> 2;
        const int cbeg = part * (BN / 4), cend = cbeg + BN / 4;
        int it = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            const int b = it & 1, u = it >> 1;
            if (!mb_wait(&acc_full[b], (unsigned)(u & 1), vfailed, a.wait_ns)) break;
            tc_fence_after();
            const Tile tl = tile_of(t, a, BN);
            const int px = tl.x0 + (m % kTW), py = tl.y0 + m / kTW;
            const bool store = px < a.w && py < a.h;
            const size_t pix = ((size_t)tl.img * a.h + (store ? py : 0)) * a.w + (store ? px : 0);
#pragma unroll 1
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0), v);
                if (!store) continue;
                const int co = tl.n0 + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float x = v[i] + (a.bias ? __ldg(a.bias + co + i) : 0.f);
                    v[i] = a.act == 1 ? silu(x) : x;
                }
                if (a.y_bf16) {
                    __nv_bfloat162 h2[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        h2[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    if (a.act == 3) {
                        // times SiLU' of the pre-activation, as k_silu_grad forms it
                        const uint4 *src = reinterpret_cast<const uint4 *>(
                            static_cast<const __nv_bfloat16 *>(a.y2) + pix * a.cout + co);
                        uint4 pp[2] = {src[0], src[1]};
                        const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(pp);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float2 g = __bfloat1622float2(h2[i]), pf = __bfloat1622float2(p2[i]);
                            h2[i] = __floats2bfloat162_rn(g.x * silu_grad_of(pf.x),
                                                          g.y * silu_grad_of(pf.y));
                        }
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.y) +
                                                           pix * a.cout + co);
                    dst[0] = *reinterpret_cast<uint4 *>(&h2[0]);
                    dst[1] = *reinterpret_cast<uint4 *>(&h2[4]);
                    if (a.act == 2) {
                        // SiLU of the rounded pre-activation, as k_silu forms it
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float2 f = __bfloat1622float2(h2[i]);
                            h2[i] = __floats2bfloat162_rn(silu_of(f.x), silu_of(f.y));
                        }
                        uint4 *dst2 = reinterpret_cast<uint4 *>(
                            static_cast<__nv_bfloat16 *>(a.y2) + pix * a.cout + co);
                        dst2[0] = *reinterpret_cast<uint4 *>(&h2[0]);
                        dst2[1] = *reinterpret_cast<uint4 *>(&h2[4]);
                    }
                } else {
                    float4 *dst =
                        reinterpret_cast<float4 *>(static_cast<float *>(a.y) + pix * a.cout + co);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
            // this warp's reads of accumulator b are complete: release it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&acc_empty[b]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *vfailed && a.status) atomicExch(a.status, (int)FWI_ERR_DEVICE_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Pixels-as-N variant for 128-channel output blocks whose width is not a
// multiple of 256: the MMA's rate per SM grows with N, so the roles swap --
// M = 128 output channels (the weight block, operand A), N = 192 output
// pixels (an 8 x 24 tile, operand B: the tap views of a 10 x 26 halo box,
// 24 groups of 8 rows 1280 bytes apart).  The accumulator holds channels in
// its lanes and pixels in its columns, so an epilogue warp (one lane quarter =
// 32 channels, a quarter of the 192 columns) stores 32 consecutive channels
// of a pixel per instruction.  Producer, MMA issuer, rings, double
// accumulators and bounded waits as in k_conv3x3_tc.
constexpr int kPW = 8, kPH = 24, kPN = kPW * kPH;          // 192 output pixels per tile
constexpr int kPHX = kPW + 2, kPHY = kPH + 2;               // halo box 10 x 26
constexpr int kPHaloTx = kPHX * kPHY * kBK * 2;             // 33,280 bytes
constexpr int kPHaloBytes = (kPHaloTx + 1023) / 1024 * 1024;
constexpr int kPM = 128;                                    // output channels per tile
constexpr int kPWBytes = kPM * kBK * 2;                     // 16 KB weight block
constexpr int kPWStages = 8;
constexpr uint32_t kPTmemCols = 512;                        // two 192-column accumulators
// bf16 epilogue staging: per epilogue warp 16 pixels x 32 channels (1 KB), so
// that a step leaves as 16-byte stores of 8 channels instead of one 2-byte
// store per channel and pixel
constexpr int kPStageBytes = 16 * 32 * 2;
constexpr int kPEpiBytes = kEpiWarps * kPStageBytes;

__host__ __device__ constexpr uint32_t idesc_bf16_mn(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ Tile tile_of_pn(int t, const ConvArgs &a)
{
    Tile r;
    const int cbk = t / a.tiles;
    t -= cbk * a.tiles;
    const int tx = t % a.tiles_x;
    t /= a.tiles_x;
    const int ty = t % a.tiles_y;
    r.img = t / a.tiles_y;
    r.x0 = tx * kPW;
    r.y0 = ty * kPH;
    r.n0 = cbk * kPM;
    return r;
}

// One 16-pixel step of a pixels-as-N epilogue warp: the staging block holds
// bf16 rows [16 pixels][32 channels, from channel c]; lane l stores chunks
// l and l + 32 (pixel chunk / 4, eight channels (chunk % 4) 8 ..) as 16-byte
// stores, pixels outside the image skipped.
__device__ __forceinline__ void pn_store_rows(const __nv_bfloat16 *stg, __nv_bfloat16 *y,
                                              const ConvArgs &a, const Tile &tl, int c0, int c,
                                              int lane)
{
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int k = lane + 32 * i, j = k >> 2, part = k & 3;
        const int m = c0 + j;
        const int px = tl.x0 + (m % kPW), py = tl.y0 + m / kPW;
        if (px >= a.w || py >= a.h) continue;
        const size_t pix = ((size_t)tl.img * a.h + py) * a.w + px;
        *reinterpret_cast<uint4 *>(y + pix * a.cout + c + part * 8) =
            *reinterpret_cast<const uint4 *>(stg + j * 32 + part * 8);
    }
}

// The reverse of pn_store_rows: rows [16 pixels][32 channels, from channel c]
// of a bf16 NHWC tensor into the staging block (pixels outside the image
// left as they are: their outputs are not stored).
__device__ __forceinline__ void pn_load_rows(__nv_bfloat16 *stg, const __nv_bfloat16 *src,
                                             const ConvArgs &a, const Tile &tl, int c0, int c,
                                             int lane)
{
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int k = lane + 32 * i, j = k >> 2, part = k & 3;
        const int m = c0 + j;
        const int px = tl.x0 + (m % kPW), py = tl.y0 + m / kPW;
        if (px >= a.w || py >= a.h) continue;
        const size_t pix = ((size_t)tl.img * a.h + py) * a.w + px;
        *reinterpret_cast<uint4 *>(stg + j * 32 + part * 8) =
            *reinterpret_cast<const uint4 *>(src + pix * a.cout + c + part * 8);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_conv3x3_tc_pn(const __grid_constant__ CUtensorMap tmx,
                    const __grid_constant__ CUtensorMap tmw, const ConvArgs a)
{
    constexpr uint32_t kIdesc = idesc_bf16_mn(kPM, kPN);
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sX = base;                              // kAStages halo boxes (operand B)
    unsigned char *sW = base + kAStages * kPHaloBytes;     // kPWStages weight blocks (operand A)
    __shared__ uint64_t x_full[kAStages], x_empty[kAStages], w_full[kPWStages], w_empty[kPWStages];
    __shared__ uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    volatile int *vfailed = &failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cbs = a.cin / kBK;
    const int total = a.tiles * (((a.cout + kPM - 1) / kPM));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mb_init(&x_full[s], 1);
            mb_init(&x_empty[s], 1);
        }
        for (int s = 0; s < kPWStages; ++s) {
            mb_init(&w_full[s], 1);
            mb_init(&w_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mb_init(&acc_full[b], 1);
            mb_init(&acc_empty[b], kEpiWarps);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(kPTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int gx = 0, gw = 0;
            int last_x[kAStages], last_w[kPWStages];
            for (int s = 0; s < kAStages; ++s) last_x[s] = -1;
            for (int s = 0; s < kPWStages; ++s) last_w[s] = -1;
            for (int t = blockIdx.x; t < total && !*vfailed; t += gridDim.x) {
                const Tile tl = tile_of_pn(t, a);
                for (int cb = 0; cb < cbs && !*vfailed; ++cb) {
                    const int sx = gx % kAStages, rx = gx / kAStages;
                    if (rx > 0 && !mb_wait(&x_empty[sx], (unsigned)((rx - 1) & 1), vfailed, a.wait_ns)) break;
                    mb_expect(&x_full[sx], kPHaloTx);
                    tma_4d(sX + sx * kPHaloBytes, &tmx, cb * kBK, tl.x0 - 1, tl.y0 - 1, tl.img,
                           &x_full[sx]);
                    last_x[sx] = gx++;
                    for (int tap = 0; tap < 9; ++tap, ++gw) {
                        const int sw = gw % kPWStages, rw = gw / kPWStages;
                        if (rw > 0 && !mb_wait(&w_empty[sw], (unsigned)((rw - 1) & 1), vfailed, a.wait_ns))
                            break;
                        if (a.withhold) continue;
                        mb_expect(&w_full[sw], kPWBytes);
                        tma_2d(sW + sw * kPWBytes, &tmw, tap * a.cin + cb * kBK, tl.n0, &w_full[sw]);
                        last_w[sw] = gw;
                    }
                }
            }
            if (*vfailed) {
                drain_loads(x_full, last_x, a.wait_ns);
                drain_loads(w_full, last_w, a.wait_ns);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int gx = 0, gw = 0, it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok && !*vfailed; t += gridDim.x, ++it) {
                const int b = it & 1, u = it >> 1;
                if (u > 0 && !mb_wait(&acc_empty[b], (unsigned)((u - 1) & 1), vfailed, a.wait_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 256);
                for (int cb = 0; cb < cbs && ok; ++cb, ++gx) {
                    const int sx = gx % kAStages, rx = gx / kAStages;
                    if (!mb_wait(&x_full[sx], (unsigned)(rx & 1), vfailed, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const unsigned char *halo = sX + sx * kPHaloBytes;
                    for (int tap = 0; tap < 9; ++tap, ++gw) {
                        const int sw = gw % kPWStages, rw = gw / kPWStages;
                        if (!mb_wait(&w_full[sw], (unsigned)(rw & 1), vfailed, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int row = (tap / 3) * kPHX + tap % 3;   // (dy + 1) 10 + dx + 1
                        const uint64_t ad = sw128_desc(sW + sw * kPWBytes, 1024);
                        const uint64_t bd = sw128_desc(halo + row * 128, kPHX * 128);
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k)
                            umma_bf16(d, ad + 2 * k, bd + 2 * k, kIdesc, (cb | tap | k) != 0);
                        umma_commit(&w_empty[sw]);
                    }
                    if (ok) umma_commit(&x_empty[sx]);
                }
                if (ok) umma_commit(&acc_full[b]);
            }
        }
    } else {
        // epilogue warps 2..17: lane quarter q = 32 output channels, and a
        // quarter of the 192 pixel columns
        __nv_bfloat16 *stg = reinterpret_cast<__nv_bfloat16 *>(
            sW + kPWStages * kPWBytes + (warp - 2) * kPStageBytes);
        const int q = warp & 3;
        const int part = (warp - 2) >> 2;
        const int cbeg = part * (kPN / 4), cend = cbeg + kPN / 4;
        int it = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            const int b = it & 1, u = it >> 1;
            if (!mb_wait(&acc_full[b], (unsigned)(u & 1), vfailed, a.wait_ns)) break;
            tc_fence_after();
            const Tile tl = tile_of_pn(t, a);
            const int co = tl.n0 + q * 32 + lane;
            // a 64-channel remainder: lanes past cout hold the zero rows of the
            // weight box and store nothing (the TMEM loads stay warp-wide)
            const bool live = co < a.cout;   // the same for all 32 lanes (cout % 64 == 0)
            const float bias = a.bias && live ? __ldg(a.bias + co) : 0.f;
#pragma unroll 1
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256 + c0), v);
                if (a.y_bf16) {
                    if (!live) continue;
                    // rows of 32 channels per pixel through the warp's staging
                    // block, then two 16-byte stores a lane (a quarter of a
                    // pixel's row each)
                    __nv_bfloat16 yb[16];
                    if (a.act == 3) {
                        // the pre-activation's rows through the staging block,
                        // then times SiLU' as k_silu_grad forms it
                        pn_load_rows(stg, static_cast<const __nv_bfloat16 *>(a.y2), a, tl, c0,
                                     tl.n0 + q * 32, lane);
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j) yb[j] = stg[j * 32 + lane];
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float g = __bfloat162float(__float2bfloat16_rn(v[j] + bias));
                            stg[j * 32 + lane] =
                                __float2bfloat16_rn(g * silu_grad_of(__bfloat162float(yb[j])));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float x = v[j] + bias;
                            yb[j] = __float2bfloat16_rn(a.act == 1 ? silu(x) : x);
                            stg[j * 32 + lane] = yb[j];
                        }
                    }
                    __syncwarp();
                    pn_store_rows(stg, static_cast<__nv_bfloat16 *>(a.y), a, tl, c0,
                                  tl.n0 + q * 32, lane);
                    if (a.act == 2) {
                        // SiLU of the rounded pre-activation, as k_silu forms it
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            stg[j * 32 + lane] = __float2bfloat16_rn(silu_of(__bfloat162float(yb[j])));
                        __syncwarp();
                        pn_store_rows(stg, static_cast<__nv_bfloat16 *>(a.y2), a, tl, c0,
                                      tl.n0 + q * 32, lane);
                    }
                    __syncwarp();
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int m = c0 + j;
                    const int px = tl.x0 + (m % kPW), py = tl.y0 + m / kPW;
                    if (!live || px >= a.w || py >= a.h) continue;
                    const size_t pix = ((size_t)tl.img * a.h + py) * a.w + px;
                    const float x = v[j] + bias;
                    static_cast<float *>(a.y)[pix * a.cout + co] = a.act == 1 ? silu(x) : x;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&acc_empty[b]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kPTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *vfailed && a.status) atomicExch(a.status, (int)FWI_ERR_DEVICE_TIMEOUT);
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int BN>
size_t conv_smem()
{
    return (size_t)kAStages * kHaloBytes + (size_t)b_stages<BN>() * BN * kBK * 2 + 1024;
}

template <int BN>
cudaError_t launch_conv(const CUtensorMap &tmx, const CUtensorMap &tmw, const ConvArgs &a,
                        cudaStream_t st)
{
    const size_t smem = conv_smem<BN>();
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent: one CTA per SM (the kernel's shared memory allows no second)
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const long long total = (long long)a.tiles * (a.cout / BN);
    const unsigned grid = (unsigned)(total < sms ? total : sms);
    k_conv3x3_tc<BN><<<grid, kThreads, smem, st>>>(tmx, tmw, a);
    return cudaGetLastError();
}

cudaError_t launch_conv_pn(const CUtensorMap &tmx, const CUtensorMap &tmw, const ConvArgs &a,
                           cudaStream_t st)
{
    const size_t smem =
        (size_t)kAStages * kPHaloBytes + (size_t)kPWStages * kPWBytes + kPEpiBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc_pn,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const long long total = (long long)a.tiles * (((a.cout + kPM - 1) / kPM));
    const unsigned grid = (unsigned)(total < sms ? total : sms);
    k_conv3x3_tc_pn<<<grid, kThreads, smem, st>>>(tmx, tmw, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores.  Over the zero-padded pixel domain q =
// (b (h + 2) + yy) wp + xx (row pitch wp = w + 2 rounded up to a multiple of
// 8, yy, xx = y + 1, x + 1 inside the image), with dP^T[co][q] and X_s^T[ci][q]
// = Xpad(q + s) staged K-major (k_stage_kmajor, s = kx - 1 for kx = 0, 1, 2),
//   dW[co][ky][kx][ci] = sum_q dP^T[co][q] X_{kx-1}^T[ci][q + (ky - 1) wp]
// is, per tap, a plain K-major GEMM: M = 128 output channels (operand A),
// N = 128 input channels of a tap, K = the padded pixels.  dP^T vanishes off
// the image, so a shifted read that leaves the image (or [0, Q): the TMA fills
// zeros) contributes nothing.  A 64-channel remainder of cin or cout loads as a
// 128-row box whose rows past the tensor read zero; the epilogue stores only
// the rows and columns inside cout x cin.  A job pairs two consecutive (tap, 128-channel
// block) units into N = 256 (the MMA's rate per SM grows with N); the K range
// is split over CTAs (job fastest in the grid, so the CTAs of one split run
// together and share the dP^T and X^T blocks in L2), each writing its FP32
// partial tile, which k_wgrad_tc_reduce then adds in split order.  Warp 0
// lane 0 issues the TMA copies, warp 1 lane 0 the MMAs, warps 2..17 read the
// accumulator; every wait is bounded as in k_conv3x3_tc.
constexpr int kGStages = 4;
constexpr int kGABytes = 128 * kBK * 2;          // 16 KB: 128 output channels x 64 pixels
constexpr int kGUBytes = 128 * kBK * 2;          // 16 KB: one unit's 128 input channels
constexpr int kGBBytes = 2 * kGUBytes;
constexpr uint32_t kGTmemCols = 256;

struct WgradTcArgs {
    unsigned long long wait_ns;
    int withhold;             // 1: issue no copies (the bounded-wait self-check)
    int cin, cout, cbs, wp;   // channels, 128-channel blocks of cin, padded row pitch
    int units, pairs, jobs;
    long long kblocks, per_split;
    float *out;            // [split][C][9][C]
    int *status;
};

// Writes rows c of one 64 x 64 output tile: tT[c][q - q0] = tile[q - q0 + k][c]
// (a transpose in shared memory, lanes along c: conflict-free 2-byte reads and
// 16-byte writes at a 144-byte pitch), then out[c][q0 ..] with 8 lanes per
// 128-byte row, so that a warp stores four whole rows.
__device__ __forceinline__ void stage_store(const __nv_bfloat16 (*tile)[72], int k,
                                            __nv_bfloat16 (*tT)[72], long long q0, long long Q,
                                            __nv_bfloat16 *__restrict__ out)
{
    for (int e = threadIdx.x; e < 512; e += 256) {
        const int cl = e & 63, j = e >> 6;
        __nv_bfloat16 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = tile[8 * j + i + k][cl];
        *reinterpret_cast<uint4 *>(&tT[cl][8 * j]) = *reinterpret_cast<uint4 *>(v);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 512; e += 256) {
        const int cl = e >> 3, j = e & 7;
        if (q0 + 8 * j < Q)
            *reinterpret_cast<uint4 *>(out + (size_t)cl * Q + q0 + 8 * j) =
                *reinterpret_cast<const uint4 *>(&tT[cl][8 * j]);
    }
}

// out[c][q] = Xpad(q + shift)[c] for q < Q (0 outside the image and [0, Q)):
// a 64 (q) x 64 (c) tile per CTA through shared memory, 16-byte loads along c
// and 16-byte stores along q
__global__ void __launch_bounds__(256)
    k_stage_kmajor(int h, int w, int C, int wp, long long Q, int shift,
                   const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out)
{
    __shared__ __align__(16) __nv_bfloat16 tile[66][72];
    __shared__ __align__(16) __nv_bfloat16 tileT[1][64][72];
    const long long q0 = (long long)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const long long img = (long long)(h + 2) * wp;
    for (int e = threadIdx.x; e < 512; e += 256) {
        const int ql = e >> 3, j = e & 7;
        const long long p = q0 + ql + shift;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p >= 0 && p < Q) {
            const long long b = p / img;
            const int r = (int)(p - b * img);
            const int yy = r / wp, xx = r - (r / wp) * wp;
            if (yy >= 1 && yy <= h && xx >= 1 && xx <= w)
                v = *reinterpret_cast<const uint4 *>(
                    in + ((b * h + (yy - 1)) * (long long)w + (xx - 1)) * C + c0 + 8 * j);
        }
        *reinterpret_cast<uint4 *>(&tile[ql][8 * j]) = v;
    }
    __syncthreads();
    stage_store(tile, 0, tileT[0], q0, Q, out + (size_t)c0 * Q);
}

__global__ void __launch_bounds__(256)
    k_stage_kmajor3(int h, int w, int C, int wp, long long Q, const __nv_bfloat16 *__restrict__ in,
                    __nv_bfloat16 *__restrict__ out0, __nv_bfloat16 *__restrict__ out1,
                    __nv_bfloat16 *__restrict__ out2)
{
    __shared__ __align__(16) __nv_bfloat16 tile[66][72];
    __shared__ __align__(16) __nv_bfloat16 tileT[3][64][72];
    const long long q0 = (long long)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const long long img = (long long)(h + 2) * wp;
    for (int e = threadIdx.x; e < 66 * 8; e += 256) {
        const int ql = e >> 3, j = e & 7;
        const long long p = q0 - 1 + ql;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p >= 0 && p < Q) {
            const long long b = p / img;
            const int r = (int)(p - b * img);
            const int yy = r / wp, xx = r - (r / wp) * wp;
            if (yy >= 1 && yy <= h && xx >= 1 && xx <= w)
                v = *reinterpret_cast<const uint4 *>(
                    in + ((b * h + (yy - 1)) * (long long)w + (xx - 1)) * C + c0 + 8 * j);
        }
        *reinterpret_cast<uint4 *>(&tile[ql][8 * j]) = v;
    }
    __syncthreads();
    stage_store(tile, 0, tileT[0], q0, Q, out0 + (size_t)c0 * Q);
    stage_store(tile, 1, tileT[1], q0, Q, out1 + (size_t)c0 * Q);
    stage_store(tile, 2, tileT[2], q0, Q, out2 + (size_t)c0 * Q);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tma, const __grid_constant__ CUtensorMap tmb0,
               const __grid_constant__ CUtensorMap tmb1, const __grid_constant__ CUtensorMap tmb2,
               const WgradTcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + kGStages * kGABytes;
    __shared__ uint64_t full[kGStages], empty[kGStages], acc_full;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    volatile int *vfailed = &failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int job = blockIdx.x % a.jobs, split = blockIdx.x / a.jobs;
    const int cot = job / a.pairs, pair = job % a.pairs;
    const int co0 = cot * 128;
    const int u0 = 2 * pair;
    const int nb = u0 + 1 < a.units ? 2 : 1;     // units in this job
    const long long k0 = (long long)split * a.per_split;
    const long long k1 = k0 + a.per_split < a.kblocks ? k0 + a.per_split : a.kblocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(&acc_full, 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(kGTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int last[kGStages];
            for (int s = 0; s < kGStages; ++s) last[s] = -1;
            int i = 0;
            for (long long kb = k0; kb < k1 && !*vfailed; ++kb, ++i) {
                const int s = i % kGStages, r = i / kGStages;
                if (r > 0 && !mb_wait(&empty[s], (unsigned)((r - 1) & 1), vfailed, a.wait_ns)) break;
                if (a.withhold) continue;
                mb_expect(&full[s], (unsigned)(kGABytes + nb * kGUBytes));
                const int q0 = (int)(kb * kBK);
                tma_2d(sA + s * kGABytes, &tma, q0, co0, &full[s]);
                for (int j = 0; j < nb; ++j) {
                    const int u = u0 + j, tap = u / a.cbs, cb = u % a.cbs;
                    const int ky = tap / 3, kx = tap % 3;
                    const CUtensorMap *mb = kx == 0 ? &tmb0 : (kx == 1 ? &tmb1 : &tmb2);
                    tma_2d(sB + s * kGBBytes + j * kGUBytes, mb, q0 + (ky - 1) * a.wp, cb * 128,
                           &full[s]);
                }
                last[s] = i;
            }
            if (*vfailed) drain_loads(full, last, a.wait_ns);
        }
    } else if (warp == 1) {
        if (lane == 0 && k0 < k1) {
            const uint32_t idesc = idesc_bf16(nb * 128);
            bool ok = true;
            int i = 0;
            for (long long kb = k0; kb < k1; ++kb, ++i) {
                const int s = i % kGStages, r = i / kGStages;
                if (!mb_wait(&full[s], (unsigned)(r & 1), vfailed, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sw128_desc(sA + s * kGABytes, 1024);
                const uint64_t bd = sw128_desc(sB + s * kGBBytes, 1024);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    umma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (i | k) != 0);
                umma_commit(&empty[s]);
            }
            if (ok) umma_commit(&acc_full);
        }
    } else {
        // warps 2..17: lane quarter q (32 output channels), a quarter of the columns
        const int q = warp & 3;
        const int co = co0 + q * 32 + lane;
        const int part = (warp - 2) >> 2;
        const int ncols = nb * 128;
        const int cbeg = part * (ncols / 4), cend = cbeg + ncols / 4;
        const bool has = k0 < k1;
        if (!has || mb_wait(&acc_full, 0u, vfailed, a.wait_ns)) {
            tc_fence_after();
            float *o = a.out + (size_t)split * 9 * a.cin * a.cout;
#pragma unroll 1
            for (int c = cbeg; c < cend; c += 16) {
                float v[16];
                if (has) {
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                const int u = u0 + c / 128, tap = u / a.cbs, cb = u % a.cbs;
                const int ci = cb * 128 + c % 128;
                // rows past cout and columns past cin came from zero-filled TMA rows
                if (co >= a.cout || ci >= a.cin) continue;
                float4 *dst = reinterpret_cast<float4 *>(o + ((size_t)co * 9 + tap) * a.cin + ci);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kGTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && *vfailed && a.status) atomicExch(a.status, (int)FWI_ERR_DEVICE_TIMEOUT);
}

// dW[e] = sum_s part[s][e], s in order
__global__ void __launch_bounds__(256)
    k_wgrad_tc_reduce(size_t n, int splits, const float *__restrict__ part, float *__restrict__ dW)
{
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (size_t)gridDim.x * 256) {
        float s = part[e];
        for (int k = 1; k < splits; ++k) s += part[(size_t)k * n + e];
        dW[e] = s;
    }
}

struct WgradTcShape {
    int wp;
    long long Q, kblocks;
    int cbs, units, pairs, jobs;
};

WgradTcShape wgrad_tc_shape(int n, int h, int w, int cin, int cout)
{
    WgradTcShape s;
    s.wp = (w + 2 + 7) / 8 * 8;
    s.Q = (long long)n * (h + 2) * s.wp;
    s.kblocks = (s.Q + kBK - 1) / kBK;
    s.cbs = (cin + 127) / 128;          // a 64-channel remainder reads zero rows past cin
    s.units = 9 * s.cbs;
    s.pairs = (s.units + 1) / 2;
    s.jobs = ((cout + 127) / 128) * s.pairs;
    return s;
}

int wgrad_tc_splits(const WgradTcShape &g, int cin, int cout, long long work_floats)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long s = sms / g.jobs;                      // one CTA per SM
    if (s < 1) s = 1;
    if (s > g.kblocks) s = g.kblocks;
    const long long fit = work_floats / (9LL * cin * cout);
    if (s > fit) s = fit;
    if (s < 1) return 1;
    const long long per = (g.kblocks + s - 1) / s;
    return (int)((g.kblocks + per - 1) / per);      // no empty range
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

fwi_status conv_call(int n, int h, int w, int cin, int cout, const void *x, const void *wt,
                     const float *bias, int act, void *y, int y_bf16, int *status, void *stream,
                     int withhold, unsigned long long wait_ns, void *y2 = nullptr)
{
    if (n < 1 || h < 1 || w < 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n, h, w must be >= 1");
    if (cin < kBK || cin % kBK != 0 || cout < 64 || cout % 64 != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG,
                                 "cin and cout must be positive multiples of 64 (cin %d, cout %d)",
                                 cin, cout);
    if (y2) {
        if ((act != 2 && act != 3) || y_bf16 != 1 || ((uintptr_t)y2 & 15))
            return fwi::record_error(FWI_ERR_INVALID_ARG,
                                     "the second tensor needs bf16 outputs, 16-byte aligned");
    } else if (act != 0 && act != 1) {
        return fwi::record_error(FWI_ERR_INVALID_ARG, "act must be 0 or 1");
    }
    if (y_bf16 != 0 && y_bf16 != 1)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "y_bf16 must be 0 or 1");
    if (!x || !wt || !y) return fwi::record_error(FWI_ERR_INVALID_ARG, "x, w and y must not be NULL");
    if (((uintptr_t)x | (uintptr_t)wt | (uintptr_t)y) & 15)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "x, w and y must be 16-byte aligned");
    // cout not a multiple of 256 runs pixels-as-N in 128-channel blocks (a
    // 64-channel remainder on zero-filled weight rows)
    const bool pn = cout % 256 != 0;
    const int TW = pn ? kPW : kTW, TH = pn ? kPH : kTH;
    const int tiles_x = (w + TW - 1) / TW, tiles_y = (h + TH - 1) / TH;
    if ((size_t)n * tiles_y * tiles_x * (cout / 64) > 0x7fffffffull ||
        (size_t)9 * cin > 0x7fffffffull ||
        (size_t)n * h * w > ((size_t)1 << 40))
        return fwi::record_error(FWI_ERR_UNSUPPORTED, "tensor too large for this library");
    auto enc = tmap_encoder();
    if (!enc) return fwi::record_error(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int BN = 256;                  // the pixels-as-M kernel: 256-channel blocks
    CUtensorMap tmx, tmw;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
        const cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)w * cin * 2,
                                       (cuuint64_t)h * w * cin * 2};
        const cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)(pn ? kPHX : kHX),
                                   (cuuint32_t)(pn ? kPHY : kHY), 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&tmx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fwi::record_error(FWI_ERR_CUDA, "tensor map of x rejected");
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)9 * cin, (cuuint64_t)cout};
        const cuuint64_t strides[1] = {(cuuint64_t)9 * cin * 2};
        // the pixels-as-N kernel reads 128-row weight blocks (rows past cout: zeros)
        const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)(pn ? kPM : BN)};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&tmw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(wt), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fwi::record_error(FWI_ERR_CUDA, "tensor map of w rejected");
    }
    ConvArgs a{wait_ns, withhold, n, h, w, cin, cout, act, y_bf16, tiles_x, tiles_y,
               n * tiles_y * tiles_x, bias, y, status, y2};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = pn ? launch_conv_pn(tmx, tmw, a, st) : launch_conv<256>(tmx, tmw, a, st);
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_conv3x3_bf16 launch: %s", cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace

extern "C" {

fwi_status fwi_conv3x3_bf16(int n, int h, int w, int cin, int cout, const void *x, const void *wt,
                            const float *bias, int act, void *y, int y_bf16, int *status,
                            void *stream)
{
    return conv_call(n, h, w, cin, cout, x, wt, bias, act, y, y_bf16, status, stream, 0, kWaitNs);
}

fwi_status fwi_conv3x3_bf16_silu(int n, int h, int w, int cin, int cout, const void *x,
                                 const void *wt, const float *bias, void *p, void *a, int *status,
                                 void *stream)
{
    if (!a) return fwi::record_error(FWI_ERR_INVALID_ARG, "a must not be NULL");
    return conv_call(n, h, w, cin, cout, x, wt, bias, 2, p, 1, status, stream, 0, kWaitNs, a);
}

fwi_status fwi_conv3x3_bf16_silu_grad(int n, int h, int w, int cin, int cout, const void *x,
                                      const void *wt, const void *p, void *dp, int *status,
                                      void *stream)
{
    if (!p) return fwi::record_error(FWI_ERR_INVALID_ARG, "p must not be NULL");
    return conv_call(n, h, w, cin, cout, x, wt, nullptr, 3, dp, 1, status, stream, 0, kWaitNs,
                     const_cast<void *>(p));
}

fwi_status fwi_conv3x3_bf16_wait_check(int n, int h, int w, int cin, int cout, const void *x,
                                       const void *wt, void *y, int y_bf16, int *status,
                                       void *stream)
{
    if (!status)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "the wait check needs a status word");
    return conv_call(n, h, w, cin, cout, x, wt, nullptr, 0, y, y_bf16, status, stream, 1,
                     kCheckWaitNs);
}

}  // extern "C"

namespace {

fwi_status wgrad_tc_call(int n, int h, int w, int cin, int cout, const void *X, const void *dP,
                         float *dW, void *stage, long long stage_bytes, float *work,
                         long long work_floats, int *status, void *stream, int withhold,
                         unsigned long long wait_ns);

}  // namespace

extern "C" {

long long fwi_conv3x3_wgrad_tc_stage_bytes(int n, int h, int w, int cin, int cout)
{
    if (n < 1 || h < 1 || w < 1 || cin < 64 || cin % 64 != 0 || cout < 64 || cout % 64 != 0)
        return 0;
    const WgradTcShape g = wgrad_tc_shape(n, h, w, cin, cout);
    return ((long long)cout + 3LL * cin) * g.Q * 2;
}

int fwi_conv3x3_wgrad_tc_splits(int n, int h, int w, int cin, int cout, long long work_floats)
{
    if (n < 1 || h < 1 || w < 1 || cin < 64 || cin % 64 != 0 || cout < 64 || cout % 64 != 0)
        return 0;
    return wgrad_tc_splits(wgrad_tc_shape(n, h, w, cin, cout), cin, cout, work_floats);
}

fwi_status fwi_conv3x3_wgrad_tc(int n, int h, int w, int cin, int cout, const void *X,
                                const void *dP, float *dW, void *stage, long long stage_bytes,
                                float *work, long long work_floats, int *status, void *stream)
{
    return wgrad_tc_call(n, h, w, cin, cout, X, dP, dW, stage, stage_bytes, work, work_floats,
                         status, stream, 0, kWaitNs);
}

fwi_status fwi_conv3x3_wgrad_tc_wait_check(int n, int h, int w, int cin, int cout, const void *X,
                                           const void *dP, float *dW, void *stage,
                                           long long stage_bytes, int *status, void *stream)
{
    if (!status)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "the wait check needs a status word");
    return wgrad_tc_call(n, h, w, cin, cout, X, dP, dW, stage, stage_bytes, nullptr, 0, status,
                         stream, 1, kCheckWaitNs);
}

}  // extern "C"

namespace {

fwi_status wgrad_tc_call(int n, int h, int w, int cin, int cout, const void *X, const void *dP,
                         float *dW, void *stage, long long stage_bytes, float *work,
                         long long work_floats, int *status, void *stream, int withhold,
                         unsigned long long wait_ns)
{
    if (n < 1 || h < 1 || w < 1 || cin < 64 || cin % 64 != 0 || cout < 64 || cout % 64 != 0)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "n, h, w >= 1 and cin, cout multiples of 64");
    if (!X || !dP || !dW || !stage)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "X, dP, dW and stage are needed");
    if (((uintptr_t)X | (uintptr_t)dP | (uintptr_t)dW | (uintptr_t)stage | (uintptr_t)work) & 15)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "all arrays must be 16-byte aligned");
    const WgradTcShape g = wgrad_tc_shape(n, h, w, cin, cout);
    if (g.Q + g.wp + kBK >= 0x7fffffffLL)
        return fwi::record_error(FWI_ERR_UNSUPPORTED, "too many pixels for one weight gradient");
    const long long need = ((long long)cout + 3LL * cin) * g.Q * 2;
    if (stage_bytes < need)
        return fwi::record_error(FWI_ERR_INVALID_ARG, "stage needs %lld bytes", need);
    const int splits = wgrad_tc_splits(g, cin, cout, work ? work_floats : 0);
    auto enc = tmap_encoder();
    if (!enc) return fwi::record_error(FWI_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // dP^T [cout][Q], then the three X^T copies [cin][Q]
    __nv_bfloat16 *arr[4];
    arr[0] = static_cast<__nv_bfloat16 *>(stage);
    for (int k = 0; k < 3; ++k) arr[1 + k] = arr[0] + (size_t)cout * g.Q + (size_t)k * cin * g.Q;
    const unsigned qt = (unsigned)((g.Q + 63) / 64);
    k_stage_kmajor<<<dim3(qt, (unsigned)(cout / 64)), 256, 0, st>>>(
        h, w, cout, g.wp, g.Q, 0, static_cast<const __nv_bfloat16 *>(dP), arr[0]);
    k_stage_kmajor3<<<dim3(qt, (unsigned)(cin / 64)), 256, 0, st>>>(
        h, w, cin, g.wp, g.Q, static_cast<const __nv_bfloat16 *>(X), arr[1], arr[2], arr[3]);
    CUtensorMap tm[4];
    for (int k = 0; k < 4; ++k) {
        const cuuint64_t dims[2] = {(cuuint64_t)g.Q, (cuuint64_t)(k == 0 ? cout : cin)};
        const cuuint64_t strides[1] = {(cuuint64_t)g.Q * 2};
        const cuuint32_t box[2] = {(cuuint32_t)kBK, 128u};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&tm[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, arr[k], dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fwi::record_error(FWI_ERR_CUDA, "tensor map of the staged operands rejected");
    }
    WgradTcArgs a;
    a.wait_ns = wait_ns;
    a.withhold = withhold;
    a.cin = cin;
    a.cout = cout;
    a.cbs = g.cbs;
    a.wp = g.wp;
    a.units = g.units;
    a.pairs = g.pairs;
    a.jobs = g.jobs;
    a.kblocks = g.kblocks;
    a.per_split = (g.kblocks + splits - 1) / splits;
    a.out = splits > 1 ? work : dW;
    a.status = status;
    const size_t smem = (size_t)kGStages * (kGABytes + kGBBytes) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) {
        k_wgrad_tc<<<(unsigned)(g.jobs * splits), kThreads, smem, st>>>(tm[0], tm[1], tm[2], tm[3],
                                                                         a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && splits > 1) {
        const size_t nw = (size_t)9 * cin * cout;
        k_wgrad_tc_reduce<<<(unsigned)((nw + 255) / 256 < 1216 ? (nw + 255) / 256 : 1216), 256, 0,
                            st>>>(nw, splits, work, dW);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fwi::record_error(FWI_ERR_CUDA, "fwi_conv3x3_wgrad_tc launch: %s",
                                 cudaGetErrorString(e));
    return FWI_OK;
}

}  // namespace
