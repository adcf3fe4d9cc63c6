"""A convolutional score model on the tensor cores, for the reverse diffusion
of Algorithms 1-2 (Sec. 3.4, 6): s(x, i) = -eps(x) / sqrt(1 - abar_i) with a
noise-prediction network eps of L 3x3 convolution layers (``channels`` wide,
SiLU between them; the input state enters as channel 0, the output is
channel 0 of the last layer; the step i enters every layer's bias as
b_l + E_l phi(i), phi sinusoidal), and its vector-Jacobian product for
Eq. chain_rule: u = (ds/dx)^T g = -(1/sqrt(1 - abar_i)) J_eps^T g.

Every step runs in the library: fwi_pack_channel0, fwi_conv3x3_bf16 (tcgen05;
bf16 activations, FP32 accumulation), fwi_silu_bf16, and for the product the
same convolution with the transposed weights W^T[ci][ky][kx][co] =
W[co][2-ky][2-kx][ci] (the adjoint of a zero-padded convolution), then
fwi_silu_grad_bf16 and fwi_unpack_channel0.  The weights are the caller's
(trained elsewhere) or seeded; this module does not train.

Use as ``Sampler(..., score_fn=ConvScore(plan.model_shape, betas))``.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import torch

from . import api


TIME_DIM = 16   # sinusoidal features of the step index


def time_features(i: int, dim: int = TIME_DIM) -> np.ndarray:
    """phi(i) = [sin(i w_k), cos(i w_k)], w_k = 10000^(-k / (dim/2)), k < dim/2."""
    k = np.arange(dim // 2, dtype=np.float64)
    w = 10000.0 ** (-k / (dim // 2))
    return np.concatenate([np.sin(i * w), np.cos(i * w)])


def seeded_weights(channels: int = 128, layers: int = 3, seed: int = 0):
    """[(W [C][3][3][C], b [C], E [C][TIME_DIM])] float32 with zero-mean normal
    entries: W of variance 1/(9 C) (1/9 for the first layer, whose input is one
    channel), b and the time projection E of standard deviation 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(layers):
        fan = 9 if l == 0 else 9 * channels
        w = rng.standard_normal((channels, 3, 3, channels)) / np.sqrt(fan)
        b = 0.1 * rng.standard_normal(channels)
        e = 0.1 * rng.standard_normal((channels, TIME_DIM))
        out.append((w.astype(np.float32), b.astype(np.float32), e.astype(np.float32)))
    return out


class ConvScore:
    """Callable score model (v_i, i) -> (s, vjp) for the Sampler."""

    def __init__(self, model_shape: Sequence[int], betas: Sequence[float], weights=None,
                 channels: int = 128, layers: int = 3, seed: int = 0, device=None):
        B, nz, nx = model_shape
        self.shape = (B, nz, nx)
        self.C = weights[0][0].shape[0] if weights is not None else channels
        self.dev = torch.device(device) if device is not None else torch.device("cuda")
        weights = weights if weights is not None else seeded_weights(channels, layers, seed)
        self.L = len(weights)
        self.abar = [None] + [api.fwi_ddpm_coefficients(list(betas), i).abar
                              for i in range(1, len(betas) + 1)]
        self.W, self.WT, self.bias = [], [], []
        steps = np.arange(len(betas) + 1)
        phi = np.stack([time_features(int(i)) for i in steps])            # [N + 1][TIME_DIM]
        for w, b, e in weights:
            w = torch.as_tensor(np.asarray(w, np.float32))
            self.W.append(w.to(torch.bfloat16).to(self.dev).contiguous())
            # W^T[ci][ky][kx][co] = W[co][2-ky][2-kx][ci]
            wt = torch.flip(w, dims=(1, 2)).permute(3, 1, 2, 0).contiguous()
            self.WT.append(wt.to(torch.bfloat16).to(self.dev))
            # per-step biases b + E phi(i) for every i, formed once in FP64
            bi = np.asarray(b, np.float64)[None, :] + phi @ np.asarray(e, np.float64).T
            self.bias.append(torch.as_tensor(bi.astype(np.float32)).to(self.dev))
        act = (B, nz, nx, self.C)
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        self.X0 = torch.empty(act, **bf)
        self.P = [torch.empty(act, **bf) for _ in range(self.L - 1)]   # pre-activations
        self.A = [torch.empty(act, **bf) for _ in range(self.L - 1)]   # activations
        self.Y = torch.empty(act, dtype=torch.float32, device=self.dev)
        self.dH = [torch.empty(act, **bf) for _ in range(2)]
        self.dX = torch.empty(act, dtype=torch.float32, device=self.dev)
        self.s = torch.empty(self.shape, dtype=torch.float32, device=self.dev)
        self.u = torch.empty(self.shape, dtype=torch.float32, device=self.dev)

    def eps(self, x: torch.Tensor, i: int, scale: float = 1.0, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
        """scale * eps(x, i) for x [B][nz][nx] (keeps the activations for vjp)."""
        api.fwi_pack_channel0(x, self.X0, 1.0, stream)
        h = self.X0
        for l in range(self.L):
            b = self.bias[l][i]
            if l < self.L - 1:
                api.fwi_conv3x3_bf16(h, self.W[l], b, 0, self.P[l], stream=stream)
                api.fwi_silu_bf16(self.P[l], self.A[l], stream)
                h = self.A[l]
            else:
                api.fwi_conv3x3_bf16(h, self.W[l], b, 0, self.Y, stream=stream)
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32,
                                                      device=self.dev)
        api.fwi_unpack_channel0(self.Y, out, scale, stream)
        return out

    def eps_vjp(self, g: torch.Tensor, scale: float = 1.0, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        """scale * J_eps(x)^T g at the x of the last eps() call."""
        api.fwi_pack_channel0(g.contiguous(), self.dH[0], scale, stream)
        d, k = self.dH[0], 0
        for l in range(self.L - 1, -1, -1):
            if l > 0:
                nxt = self.dH[1 - k]
                api.fwi_conv3x3_bf16(d, self.WT[l], None, 0, nxt, stream=stream)
                api.fwi_silu_grad_bf16(nxt, self.P[l - 1], nxt, stream)
                d, k = nxt, 1 - k
            else:
                api.fwi_conv3x3_bf16(d, self.WT[0], None, 0, self.dX, stream=stream)
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32,
                                                      device=self.dev)
        api.fwi_unpack_channel0(self.dX, out, 1.0, stream)
        return out

    def __call__(self, v_i: torch.Tensor, i: int):
        c = -1.0 / float(np.sqrt(1.0 - self.abar[i]))
        s = self.eps(v_i, i, c, self.s)

        def vjp(g):
            return self.eps_vjp(g, c, self.u)

        return s, vjp
