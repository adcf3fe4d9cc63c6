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
fwi_silu_grad_bf16 and fwi_unpack_channel0.  The weights are the caller's,
seeded, or trained here by denoising score matching (DSMTrainer, Eq.
L2_rewrite): the network keeps FP32 master parameters in one flat buffer
and refreshes its bf16 weights, their transposes and the per-step bias
tables from them with fwi_conv3x3_weights_prep and fwi_time_bias.

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
        C, N1 = self.C, len(betas) + 1
        # FP32 master parameters [(W_l, b_l, E_l)] as views of one flat buffer
        sizes = [C * 9 * C, C, C * TIME_DIM]
        self.theta = torch.empty(self.L * sum(sizes), dtype=torch.float32, device=self.dev)
        self.params = self.layer_views(self.theta)
        for (w, b, e), views in zip(weights, self.params):
            for src, dst in zip((w, b, e), views):
                dst.copy_(torch.as_tensor(np.asarray(src, np.float32)))
        self.phi = torch.tensor(np.stack([time_features(i) for i in range(N1)]),
                                dtype=torch.float32, device=self.dev)     # [N + 1][TIME_DIM]
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        self.W = [torch.empty((C, 3, 3, C), **bf) for _ in range(self.L)]
        self.WT = [torch.empty((C, 3, 3, C), **bf) for _ in range(self.L)]
        self.bias = [torch.empty((N1, C), dtype=torch.float32, device=self.dev)
                     for _ in range(self.L)]
        self.refresh()
        act = (B, nz, nx, self.C)
        self.X0 = torch.empty(act, **bf)
        self.P = [torch.empty(act, **bf) for _ in range(self.L - 1)]   # pre-activations
        self.A = [torch.empty(act, **bf) for _ in range(self.L - 1)]   # activations
        self.Y = torch.empty(act, dtype=torch.float32, device=self.dev)
        self.dH = [torch.empty(act, **bf) for _ in range(2)]
        self.dX = torch.empty(act, dtype=torch.float32, device=self.dev)
        self.s = torch.empty(self.shape, dtype=torch.float32, device=self.dev)
        self.u = torch.empty(self.shape, dtype=torch.float32, device=self.dev)

    def layer_views(self, flat: torch.Tensor):
        """[(W [C][3][3][C], b [C], E [C][TIME_DIM])] views of a flat buffer
        laid out like ``theta``."""
        C, out, o = self.C, [], 0
        for _ in range(self.L):
            shapes = ((C, 3, 3, C), (C,), (C, TIME_DIM))
            views = []
            for sh in shapes:
                n = int(np.prod(sh))
                views.append(flat[o:o + n].view(sh))
                o += n
            out.append(tuple(views))
        return out

    def refresh(self, stream=None):
        """bf16 W, W^T[ci][ky][kx][co] = W[co][2-ky][2-kx][ci] and the per-step
        biases b + E phi(i) of every layer, from the FP32 master parameters."""
        for l, (w, b, e) in enumerate(self.params):
            api.fwi_conv3x3_weights_prep(w, self.W[l], self.WT[l], stream)
            api.fwi_time_bias(b, e, self.phi, self.bias[l], stream)

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

    def param_grads(self, g: torch.Tensor, i: int, grads, work: torch.Tensor | None = None,
                    stage: torch.Tensor | None = None, stream=None):
        """The gradient of <eps(x, i), g> with respect to every (W, b, E),
        written into ``grads`` (layer_views of a flat buffer), at the x of the
        last eps() call: per layer the weight gradient from the layer's input
        and its output gradient (fwi_conv3x3_wgrad), the bias gradient
        (fwi_channel_sum) and E's (fwi_time_bias_grad), then the output
        gradient of the layer below as in eps_vjp.  ``work``: float32 scratch
        for the weight gradient's partial sums; with ``stage`` (the K-major
        staging buffer, channels a multiple of 128) the weight gradient runs on
        the tensor cores (api.fwi_conv3x3_wgrad_tc), else on the CUDA cores
        (api.fwi_conv3x3_wgrad)."""
        api.fwi_pack_channel0(g.contiguous(), self.dH[0], 1.0, stream)
        d, k = self.dH[0], 0
        for l in range(self.L - 1, -1, -1):
            dW, db, dE = grads[l]
            src = self.X0 if l == 0 else self.A[l - 1]
            if stage is not None:
                api.fwi_conv3x3_wgrad_tc(src, d, dW, stage, work, stream=stream)
            else:
                api.fwi_conv3x3_wgrad(src, d, dW, work, stream)
            api.fwi_channel_sum(d, db, work, stream)
            api.fwi_time_bias_grad(db, self.phi[i], dE, stream)
            if l > 0:
                nxt = self.dH[1 - k]
                api.fwi_conv3x3_bf16(d, self.WT[l], None, 0, nxt, stream=stream)
                api.fwi_silu_grad_bf16(nxt, self.P[l - 1], nxt, stream)
                d, k = nxt, 1 - k

    def __call__(self, v_i: torch.Tensor, i: int):
        c = -1.0 / float(np.sqrt(1.0 - self.abar[i]))
        s = self.eps(v_i, i, c, self.s)

        def vjp(g):
            return self.eps_vjp(g, c, self.u)

        return s, vjp


class DSMTrainer:
    """Denoising score matching (Eq. L2_rewrite) of a ConvScore with Adam.

    One step on a minibatch x_0 [B][nz][nx] (normalised models), its noise z
    and one step index t (every sample of the minibatch shares t): x_t =
    sqrt(abar_t) x_0 + sqrt(1 - abar_t) z (fwi_dsm_noisy), eps(x_t, t), the loss
    mean (eps - z)^2 and its gradient (fwi_dsm_loss) -- the integrand of Eq.
    L2_rewrite for s = -eps / sqrt(1 - abar) weighted by kappa = 1 - abar --
    the parameter gradients (ConvScore.param_grads), one Adam step over the
    flat FP32 parameters (fwi_adam_step) and the refresh of the bf16 weights
    and bias tables.  ``step`` returns the loss as a device scalar."""

    def __init__(self, net: ConvScore, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        self.net, self.lr, self.beta1, self.beta2, self.eps_adam = net, lr, beta1, beta2, eps
        f32 = dict(dtype=torch.float32, device=net.dev)
        self.grad = torch.zeros_like(net.theta)
        self.m = torch.zeros_like(net.theta)
        self.v = torch.zeros_like(net.theta)
        self.grads = net.layer_views(self.grad)
        self.xt = torch.empty(net.shape, **f32)
        self.e = torch.empty(net.shape, **f32)
        self.g = torch.empty(net.shape, **f32)
        self.loss = torch.empty((1,), **f32)
        self.work = torch.empty(api.WGRAD_MAX_SPLITS * 9 * net.C * net.C, **f32)
        # the K-major staging buffer of the tensor-core weight gradient
        self.stage = None
        if net.C % 128 == 0:
            nbytes = api.fwi_conv3x3_wgrad_tc_stage_bytes(*net.shape, net.C)
            self.stage = torch.empty(nbytes, dtype=torch.uint8, device=net.dev)
        self.k = 0

    def gradients(self, x0: torch.Tensor, z: torch.Tensor, t: int, stream=None) -> torch.Tensor:
        """The loss of the minibatch at step t and its gradient in ``grad``."""
        net = self.net
        if not 1 <= t < len(net.abar):
            raise ValueError(f"step {t} outside 1..{len(net.abar) - 1}")
        api._f32(x0, net.shape, "x0")
        api._f32(z, net.shape, "z")
        api.fwi_dsm_noisy(x0, z, net.abar[t], self.xt, stream)
        net.eps(self.xt, t, 1.0, self.e, stream)
        api.fwi_dsm_loss(self.e, z, self.loss, self.g, self.work, stream)
        net.param_grads(self.g, t, self.grads, self.work, self.stage, stream)
        return self.loss

    def step(self, x0: torch.Tensor, z: torch.Tensor, t: int, stream=None) -> torch.Tensor:
        loss = self.gradients(x0, z, t, stream)
        self.k += 1
        api.fwi_adam_step(self.net.theta, self.grad, self.m, self.v, self.k, self.lr, self.beta1,
                          self.beta2, self.eps_adam, stream)
        self.net.refresh(stream)
        return loss
