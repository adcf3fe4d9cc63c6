"""A convolutional score model on the tensor cores, for the reverse diffusion
of Algorithms 1-2 (Sec. 3.4, 6): s(x, i) = -eps(x) / sqrt(1 - abar_i) with a
noise-prediction network eps of L 3x3 convolution layers (``channels`` wide,
SiLU between them; the input state enters as channel 0, the output is
channel 0 of the last layer; the step i enters every layer's bias as
b_l + E_l phi(i), phi sinusoidal), and its vector-Jacobian product for
Eq. chain_rule: u = (ds/dx)^T g = -(1/sqrt(1 - abar_i)) J_eps^T g.

Every step runs in the library: fwi_pack_channel0, fwi_conv3x3_bf16_silu
(tcgen05; bf16 activations, FP32 accumulation; the pre-activation and its
SiLU written by one epilogue; the U-Net runs fwi_conv3x3_bf16 and
fwi_silu_bf16), fwi_conv3x3_bf16 for the last layer, and for the product the
same convolution with the transposed weights W^T[ci][ky][kx][co] =
W[co][2-ky][2-kx][ci] (the adjoint of a zero-padded convolution) times SiLU'
in its epilogue (fwi_conv3x3_bf16_silu_grad; the U-Net runs
fwi_silu_grad_bf16 on its summed gradients), then fwi_unpack_channel0.  The
weights are the caller's, seeded, or trained here by denoising score
matching (DSMTrainer, Eq.
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

    def work_floats(self) -> int:
        return api.WGRAD_MAX_SPLITS * 9 * self.C * self.C

    def stage_bytes(self) -> int:
        return api.fwi_conv3x3_wgrad_tc_stage_bytes(*self.shape, self.C, self.C)

    def refresh(self, stream=None):
        """bf16 W, W^T[ci][ky][kx][co] = W[co][2-ky][2-kx][ci] and the per-step
        biases b + E phi(i) of every layer, from the FP32 master parameters."""
        for l, (w, b, e) in enumerate(self.params):
            api.fwi_conv3x3_weights_prep(w, self.W[l], self.WT[l], stream)
            api.fwi_time_bias(b, e, self.phi, self.bias[l], stream)

    def eps(self, x: torch.Tensor, i: int, scale: float = 1.0, out: torch.Tensor | None = None,
            stream=None, in_scale: float = 1.0) -> torch.Tensor:
        """scale * eps(in_scale x, i) for x [B][nz][nx] (keeps the activations for vjp)."""
        api.fwi_pack_channel0(x, self.X0, in_scale, stream)
        h = self.X0
        for l in range(self.L):
            b = self.bias[l][i]
            if l < self.L - 1:
                api.fwi_conv3x3_bf16_silu(h, self.W[l], b, self.P[l], self.A[l], stream=stream)
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
                api.fwi_conv3x3_bf16_silu_grad(d, self.WT[l], self.P[l - 1], nxt, stream=stream)
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
        staging buffer) the weight gradient runs on the tensor cores
        (api.fwi_conv3x3_wgrad_tc), else on the CUDA cores
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
                api.fwi_conv3x3_bf16_silu_grad(d, self.WT[l], self.P[l - 1], nxt, stream=stream)
                d, k = nxt, 1 - k

    def __call__(self, v_i: torch.Tensor, i: int):
        c = -1.0 / float(np.sqrt(1.0 - self.abar[i]))
        s = self.eps(v_i, i, c, self.s)

        def vjp(g):
            return self.eps_vjp(g, c, self.u)

        return s, vjp


class DSMTrainer:
    """Denoising score matching (Eq. L2_rewrite) of a ConvScore or UNetScore
    with Adam.

    One step on a minibatch x_0 [B][nz][nx] (normalised models), its noise z
    and one step index t (every sample of the minibatch shares t): x_t =
    sqrt(abar_t) x_0 + sqrt(1 - abar_t) z (fwi_dsm_noisy), eps(x_t, t), the loss
    mean (eps - z)^2 and its gradient (fwi_dsm_loss) -- the integrand of Eq.
    L2_rewrite for s = -eps / sqrt(1 - abar) weighted by kappa = 1 - abar --
    the parameter gradients (ConvScore.param_grads), one Adam step over the
    flat FP32 parameters (fwi_adam_step) and the refresh of the bf16 weights
    and bias tables.  ``step`` returns the loss as a device scalar.
    ``regression_step`` trains the same network on supervised pairs instead
    (a network surrogate of the physics gradient, sampler.NetworkSurrogate)."""

    def __init__(self, net, lr: float = 1e-3, beta1: float = 0.9,
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
        self.work = torch.empty(net.work_floats(), **f32)
        # the K-major staging buffer of the tensor-core weight gradient
        nbytes = net.stage_bytes()
        self.stage = torch.empty(nbytes, dtype=torch.uint8, device=net.dev) if nbytes else None
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

    def regression_gradients(self, x: torch.Tensor, y: torch.Tensor, i: int = 0,
                             in_scale: float = 1.0, stream=None) -> torch.Tensor:
        """Supervised regression of the network on pairs (x, y), both
        [B][nz][nx]: the loss mean (eps(in_scale x, i) - y)^2 (the same
        fwi_dsm_loss) and its gradient in ``grad``; i selects the bias row
        (0 for a network that is not step-conditioned)."""
        net = self.net
        api._f32(x, net.shape, "x")
        api._f32(y, net.shape, "y")
        net.eps(x, i, 1.0, self.e, stream, in_scale=in_scale)
        api.fwi_dsm_loss(self.e, y, self.loss, self.g, self.work, stream)
        net.param_grads(self.g, i, self.grads, self.work, self.stage, stream)
        return self.loss

    def regression_step(self, x: torch.Tensor, y: torch.Tensor, i: int = 0,
                        in_scale: float = 1.0, stream=None) -> torch.Tensor:
        loss = self.regression_gradients(x, y, i, in_scale, stream)
        self._update(stream)
        return loss

    def _update(self, stream=None):
        self.k += 1
        api.fwi_adam_step(self.net.theta, self.grad, self.m, self.v, self.k, self.lr, self.beta1,
                          self.beta2, self.eps_adam, stream)
        self.net.refresh(stream)

    def step(self, x0: torch.Tensor, z: torch.Tensor, t: int, stream=None) -> torch.Tensor:
        loss = self.gradients(x0, z, t, stream)
        self.k += 1
        api.fwi_adam_step(self.net.theta, self.grad, self.m, self.v, self.k, self.lr, self.beta1,
                          self.beta2, self.eps_adam, stream)
        self.net.refresh(stream)
        return loss


# --------------------------------------------------------------------------
# A 4-level U-Net noise-prediction network (the score model of Sec. 6 is a
# U-Net; no architecture is given): level widths c_0..c_3, two 3x3
# convolution + SiLU layers per encoder level with 2 x 2 mean pooling between
# levels, and per decoder level nearest upsampling, a convolution + SiLU, the
# additive skip from the encoder layer of that level and a second convolution
# + SiLU; a last linear convolution whose channel 0 is eps.  The step enters
# every layer's bias as b + E phi(i).

UNET_WIDTHS = (32, 64, 128, 256)


def unet_layers(widths=UNET_WIDTHS):
    """[(name, level, cin, cout)] of the U-Net's convolutions, in parameter order."""
    c = tuple(widths)
    if len(c) != 4 or any(w < 32 or w % 32 for w in c):
        raise ValueError("four level widths, each a multiple of 32")
    out = []
    for k in range(4):
        out += [(f"enc{k}a", k, c[0] if k == 0 else c[k - 1], c[k]), (f"enc{k}b", k, c[k], c[k])]
    for k in (2, 1, 0):
        out += [(f"dec{k}u", k, c[k + 1], c[k]), (f"dec{k}c", k, c[k], c[k])]
    out.append(("out", 0, c[0], c[0]))
    return out


def unet_block_widths(widths=UNET_WIDTHS):
    """The widths the tensor-core convolution computes with: each rounded up to
    its 64-channel blocks.  A level of 32 channels runs as 64 whose last 32
    channels hold zeros -- weights, biases and step embeddings into and out of
    them are zero, so their activations are SiLU(0) = 0 and every gradient
    reaching their parameters is exactly zero: the network computed is the
    32-channel one."""
    return tuple(-(-int(w) // 64) * 64 for w in widths)


def unet_embed(weights, widths, block_widths):
    """Logical weights [(W, b, E)] of ``widths`` placed into the leading
    channels of zero arrays of ``block_widths``."""
    out = []
    for (W, b, E), (_, _, ci, co), (_, _, cb, ob) in zip(weights, unet_layers(widths),
                                                          unet_layers(block_widths)):
        Wp = np.zeros((ob, 3, 3, cb), np.float32)
        bp = np.zeros(ob, np.float32)
        Ep = np.zeros((ob, TIME_DIM), np.float32)
        Wp[:co, :, :, :ci] = W
        bp[:co] = b
        Ep[:co] = E
        out.append((Wp, bp, Ep))
    return out


def unet_seeded_weights(widths=UNET_WIDTHS, seed: int = 0):
    """[(W [cout][3][3][cin], b [cout], E [cout][TIME_DIM])] float32, W of
    variance 1/(9 cin) (1/9 for the first layer, whose input is one channel),
    b and E of standard deviation 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for name, _, cin, cout in unet_layers(widths):
        fan = 9 if name == "enc0a" else 9 * cin
        w = rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(fan)
        b = 0.1 * rng.standard_normal(cout)
        e = 0.1 * rng.standard_normal((cout, TIME_DIM))
        out.append((w.astype(np.float32), b.astype(np.float32), e.astype(np.float32)))
    return out


class UNetScore:
    """Callable score model (v_i, i) -> (s, vjp) for the Sampler, and a
    network DSMTrainer can train: the 4-level U-Net above on the library's
    kernels (tcgen05 convolutions, fwi_pool2_bf16, fwi_up2_bf16, fwi_add_bf16,
    SiLU kernels), bf16 activations and gradients, FP32 master parameters."""

    def __init__(self, model_shape: Sequence[int], betas: Sequence[float], weights=None,
                 widths=UNET_WIDTHS, seed: int = 0, device=None):
        B, nz, nx = model_shape
        self.shape = (B, nz, nx)
        self.logical_widths = tuple(widths)
        self.logical_layers = unet_layers(widths)
        self.widths = unet_block_widths(widths)      # what the kernels compute with
        self.layers = unet_layers(self.widths)
        self.idx = {name: l for l, (name, _, _, _) in enumerate(self.layers)}
        self.L = len(self.layers)
        self.dev = torch.device(device) if device is not None else torch.device("cuda")
        weights = weights if weights is not None else unet_seeded_weights(widths, seed)
        if len(weights) != self.L:
            raise ValueError(f"the U-Net has {self.L} layers")
        weights = unet_embed(weights, widths, self.widths)
        self.abar = [None] + [api.fwi_ddpm_coefficients(list(betas), i).abar
                              for i in range(1, len(betas) + 1)]
        self.sizes = [(nz, nx)]
        for _ in range(3):
            h, w = self.sizes[-1]
            self.sizes.append(((h + 1) // 2, (w + 1) // 2))
        N1 = len(betas) + 1
        shapes = [((co, 3, 3, ci), (co,), (co, TIME_DIM)) for _, _, ci, co in self.layers]
        self._shapes = shapes
        self.theta = torch.empty(sum(int(np.prod(s)) for sh in shapes for s in sh),
                                 dtype=torch.float32, device=self.dev)
        self.params = self.layer_views(self.theta)
        for (w, b, e), views in zip(weights, self.params):
            for src, dst in zip((w, b, e), views):
                dst.copy_(torch.as_tensor(np.asarray(src, np.float32)))
        self.phi = torch.tensor(np.stack([time_features(i) for i in range(N1)]),
                                dtype=torch.float32, device=self.dev)
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        self.W = [torch.empty(sh[0], **bf) for sh in shapes]
        self.WT = [torch.empty((sh[0][3], 3, 3, sh[0][0]), **bf) for sh in shapes]
        self.bias = [torch.empty((N1, sh[1][0]), dtype=torch.float32, device=self.dev)
                     for sh in shapes]
        self.refresh()

        def act(k, c, dtype=torch.bfloat16):
            h, w = self.sizes[k]
            return torch.empty((B, h, w, c), dtype=dtype, device=self.dev)

        c = self.widths
        self.X0 = act(0, c[0])
        self.P = {n: act(k, co) for n, k, _, co in self.layers if n != "out"}
        self.A = {n: act(k, co) for n, k, _, co in self.layers if n != "out"}
        self.D = {k: act(k, c[k - 1]) for k in (1, 2, 3)}         # pooled encoder inputs
        self.U = {k: act(k, c[k + 1]) for k in (0, 1, 2)}         # upsampled decoder inputs
        self.S = {k: act(k, c[k]) for k in (0, 1, 2)}             # after the additive skip
        self.Y = act(0, c[0], torch.float32)
        self.dP = {n: act(k, co) for n, k, _, co in self.layers}
        self.dIn = {n: act(k, ci) for n, k, ci, _ in self.layers if n != "enc0a"}
        self.dUp = {k: act(k, c[k]) for k in (1, 2, 3)}           # d/d(an up2 input)
        self.dAcc = {k: act(k, c[k]) for k in (0, 1, 2)}          # encoder output: pool + skip
        self.dPool = {k: act(k, c[k]) for k in (0, 1, 2)}         # d/d(a pool2 input)
        self.dX = act(0, c[0], torch.float32)
        self.s = torch.empty(self.shape, dtype=torch.float32, device=self.dev)
        self.u = torch.empty(self.shape, dtype=torch.float32, device=self.dev)

    def logical(self, views):
        """The network's own parameters (or their gradients) out of per-layer
        (W, b, E) views of the block widths: the leading channels."""
        return [(W[:co, :, :, :ci], b[:co], E[:co])
                for (W, b, E), (_, _, ci, co) in zip(views, self.logical_layers)]

    # the interface DSMTrainer uses
    def layer_views(self, flat: torch.Tensor):
        out, o = [], 0
        for sh in self._shapes:
            views = []
            for s in sh:
                n = int(np.prod(s))
                views.append(flat[o:o + n].view(s))
                o += n
            out.append(tuple(views))
        return out

    def work_floats(self) -> int:
        return api.WGRAD_MAX_SPLITS * 9 * max(ci * co for _, _, ci, co in self.layers)

    def stage_bytes(self) -> int:
        B = self.shape[0]
        return max(api.fwi_conv3x3_wgrad_tc_stage_bytes(B, *self.sizes[k], ci, co)
                   for _, k, ci, co in self.layers)

    def refresh(self, stream=None):
        for l, (w, b, e) in enumerate(self.params):
            api.fwi_conv3x3_weights_prep(w, self.W[l], self.WT[l], stream)
            api.fwi_time_bias(b, e, self.phi, self.bias[l], stream)

    def _conv(self, name, x, i, stream):
        l = self.idx[name]
        # two passes here: with the U-Net's many small 64-channel layers the
        # fused epilogue measured no faster (6.22 against 6.15 ms a DSM step)
        api.fwi_conv3x3_bf16(x, self.W[l], self.bias[l][i], 0, self.P[name], stream=stream)
        api.fwi_silu_bf16(self.P[name], self.A[name], stream)
        return self.A[name]

    def eps(self, x: torch.Tensor, i: int, scale: float = 1.0, out: torch.Tensor | None = None,
            stream=None, in_scale: float = 1.0) -> torch.Tensor:
        """scale * eps(in_scale x, i) for x [B][nz][nx] (keeps the activations for
        the backward pass)."""
        api.fwi_pack_channel0(x, self.X0, in_scale, stream)
        h = self.X0
        for k in range(4):
            if k > 0:
                api.fwi_pool2_bf16(h, self.D[k], 0, stream)
                h = self.D[k]
            h = self._conv(f"enc{k}a", h, i, stream)
            h = self._conv(f"enc{k}b", h, i, stream)
        for k in (2, 1, 0):
            api.fwi_up2_bf16(h, self.U[k], 0, stream)
            a = self._conv(f"dec{k}u", self.U[k], i, stream)
            api.fwi_add_bf16(a, self.A[f"enc{k}b"], self.S[k], stream)
            h = self._conv(f"dec{k}c", self.S[k], i, stream)
        l = self.idx["out"]
        api.fwi_conv3x3_bf16(h, self.W[l], self.bias[l][i], 0, self.Y, stream=stream)
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32,
                                                      device=self.dev)
        api.fwi_unpack_channel0(self.Y, out, scale, stream)
        return out

    def _layer_back(self, name, d, src, i, grads, work, stage, stream, act=True, dst=None):
        """Through one layer from the gradient d at its output: SiLU', the
        parameter gradients (if ``grads``), and the gradient at its input
        (into ``dst`` or dIn[name]; skipped when dst is False)."""
        l = self.idx[name]
        dp = self.dP[name]
        if act:
            api.fwi_silu_grad_bf16(d, self.P[name], dp, stream)
        if grads is not None:
            dW, db, dE = grads[l]
            _, _, ci, co = self.layers[l]
            if stage is not None:
                api.fwi_conv3x3_wgrad_tc(src, dp, dW, stage, work, stream=stream)
            else:
                api.fwi_conv3x3_wgrad(src, dp, dW, work, stream)
            api.fwi_channel_sum(dp, db, work, stream)
            api.fwi_time_bias_grad(db, self.phi[i], dE, stream)
        if dst is False:
            return None
        dst = self.dIn[name] if dst is None else dst
        api.fwi_conv3x3_bf16(dp, self.WT[l], None, 0, dst, stream=stream)
        return dst

    def _backward(self, g, scale, i, grads=None, work=None, stage=None, need_input=True,
                  stream=None):
        api.fwi_pack_channel0(g.contiguous(), self.dP["out"], scale, stream)
        d = self._layer_back("out", None, self.A["dec0c"], i, grads, work, stage, stream,
                             act=False)
        for k in (0, 1, 2):
            ds = self._layer_back(f"dec{k}c", d, self.S[k], i, grads, work, stage, stream)
            du = self._layer_back(f"dec{k}u", ds, self.U[k], i, grads, work, stage, stream)
            api.fwi_pool2_bf16(du, self.dUp[k + 1], 1, stream)      # the adjoint of up2
            d = self.dUp[k + 1]
        for k in (3, 2, 1, 0):
            if k < 3:      # the encoder output also feeds the skip of its level
                api.fwi_add_bf16(d, self.dIn[f"dec{k}c"], self.dAcc[k], stream)
                d = self.dAcc[k]
            da = self._layer_back(f"enc{k}b", d, self.A[f"enc{k}a"], i, grads, work, stage,
                                  stream)
            if k > 0:
                dd = self._layer_back(f"enc{k}a", da, self.D[k], i, grads, work, stage, stream)
                api.fwi_up2_bf16(dd, self.dPool[k - 1], 1, stream)   # the adjoint of pool2
                d = self.dPool[k - 1]
            else:
                self._layer_back("enc0a", da, self.X0, i, grads, work, stage, stream,
                                 dst=self.dX if need_input else False)

    def eps_vjp(self, g: torch.Tensor, scale: float = 1.0, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        """scale * J_eps(x)^T g at the x of the last eps() call."""
        self._backward(g, scale, None, stream=stream)
        out = out if out is not None else torch.empty(self.shape, dtype=torch.float32,
                                                      device=self.dev)
        api.fwi_unpack_channel0(self.dX, out, 1.0, stream)
        return out

    def param_grads(self, g: torch.Tensor, i: int, grads, work: torch.Tensor | None = None,
                    stage: torch.Tensor | None = None, stream=None):
        """The gradient of <eps(x, i), g> with respect to every (W, b, E) into
        ``grads`` (layer_views of a flat buffer), at the x of the last eps()."""
        self._backward(g, 1.0, i, grads, work, stage, need_input=False, stream=stream)

    def __call__(self, v_i: torch.Tensor, i: int):
        c = -1.0 / float(np.sqrt(1.0 - self.abar[i]))
        s = self.eps(v_i, i, c, self.s)

        def vjp(g):
            return self.eps_vjp(g, c, self.u)

        return s, vjp
