// silu.cuh -- SiLU and its derivative as the score networks apply them to a
// bf16 pre-activation p (widened to float): silu(p) = p sigmoid(p),
// silu'(p) = sg (1 + p (1 - sg)) with sg = sigmoid(p) = 1 / (1 + e^-p).  The
// standalone elementwise kernels (score_net.cu) and the convolution's fused
// epilogue (conv_tc.cu) share these, so both give the same bits.
#pragma once

#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ float silu_sigmoid(float p) { return 1.f / (1.f + __expf(-p)); }
__device__ __forceinline__ float silu_of(float p) { return p * silu_sigmoid(p); }
__device__ __forceinline__ float silu_grad_of(float p)
{
    const float sg = silu_sigmoid(p);
    return sg * (1.f + p * (1.f - sg));
}

}  // namespace
