"""Learned forward surrogate on the library's kernels: a convolutional
encoder-decoder from a velocity model to the seismograms of the FD solver,
trained on pairs the FD solver itself generates.  It is the surrogate route
to cheaper guidance that Sec. 7 proposes: in the early, high-noise reverse
steps of Algorithm 2 (Sec. 5.2) its W2 guidance gradient -- the W2 adjoint
source of its predicted data (Eq. final_objective, fwi_w2_misfit) carried
back through the network's vector-Jacobian product -- stands in for the FD
gradient, and the FD solver stays both the check of that gradient's error and
the fallback (GatedSurrogate).

Network (every step runs in the CUDA library; bf16 activations and weights,
FP32 accumulation and master parameters):
  input   model b is column (b mod m) of image (b / m), an image being nx
          pixels high (the model's columns x) and m pixels wide; channel
          z < nz of pixel x holds (v[z][x] - 3000) / 1500, the channels above
          fixed geometry features (per shot the offset (x - x_s)/nx and its
          magnitude, a constant 1), fwi_sur_pack
  layers  six convolutions with three taps along the image (the horizontal
          taps of the tensor-core 3 x 3 convolution fixed at zero, so the m
          models of an image never mix): enc0 -> mean pooling by 4 (two
          poolings of row pairs) -> enc1 -> pooling by 4 -> enc2 (5 pixels for
          70 columns: the bottleneck sees the whole model, as the reflections
          from midpoints up to half the spread away need) -> nearest
          upsampling by 4 -> dec1 + enc1 -> upsampling by 4 -> dec0 + enc0 ->
          out; SiLU after all but ``out``
  output  Y[x][s nt + t], and the trace of receiver r (column rec_ix[r]) is
          amp sign(y) (e^|y| - 1), fwi_sur_traces; training fits Y to
          sign(d) log(1 + |d| / amp) of the FD data (fwi_sur_target,
          fwi_sur_loss), which gives weak arrivals weight as the W2 weighting
          does
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np
import torch

from . import api

LAYERS = ("enc0", "enc1", "enc2", "dec1", "dec0", "out")


def layer_table(c0: int, width: int, cout: int):
    """[(name, level, cin, cout)] of the six convolutions, in parameter order."""
    return [("enc0", 0, c0, width), ("enc1", 1, width, width), ("enc2", 2, width, width),
            ("dec1", 1, width, width), ("dec0", 0, width, width), ("out", 0, width, cout)]


def geometry_channels(nz: int, nx: int, src_ix: Sequence[int], c0: int) -> np.ndarray:
    """G [nx][c0] float32: zero below channel nz; per shot s the offset
    (x - src_ix[s]) / nx (channel nz + 2 s) and its magnitude (nz + 2 s + 1);
    then 1 (nz + 2 ns).  A fixed encoding of the acquisition the network's
    convolutions cannot infer from the velocity alone."""
    ns = len(src_ix)
    if nz + 2 * ns + 1 > c0:
        raise ValueError("c0 too small for nz + 2 ns + 1 input channels")
    G = np.zeros((nx, c0), np.float32)
    x = np.arange(nx, dtype=np.float64)
    for s, sx in enumerate(src_ix):
        G[:, nz + 2 * s] = (x - sx) / nx
        G[:, nz + 2 * s + 1] = np.abs(x - sx) / nx
    G[:, nz + 2 * ns] = 1.0
    return G


def seeded_weights(c0: int, width: int, cout: int, seed: int = 0):
    """[(W3 [cout][3][cin], b [cout])] float32: W3 of variance 1/(3 cin), the
    output layer's a sixteenth of that, biases zero."""
    rng = np.random.default_rng(seed)
    out = []
    for name, _, ci, co in layer_table(c0, width, cout):
        w = rng.standard_normal((co, 3, ci)) / np.sqrt(3 * ci)
        if name == "out":
            w /= 4.0
        out.append((w.astype(np.float32), np.zeros(co, np.float32)))
    return out


class ForwardSurrogate:
    """The network for ``nmod`` models of nz x nx on an acquisition of shots at
    columns src_ix and receivers at the distinct columns rec_ix (all on the
    surface rows the FD data record), nt samples per trace."""

    def __init__(self, nmod: int, nz: int, nx: int, nt: int, src_ix: Sequence[int],
                 rec_ix: Sequence[int], amp: float, *, width: int = 256, c0: int = 128,
                 m: int = 8, in_scale: float = 1.0 / 1500.0, in_shift: float = -2.0,
                 weights=None, seed: int = 0, device=None):
        if len(set(int(r) for r in rec_ix)) != len(rec_ix):
            raise ValueError("the surrogate needs receivers at distinct columns")
        if not all(0 <= int(c) < nx for c in list(rec_ix) + list(src_ix)):
            raise ValueError("source and receiver columns must lie in [0, nx)")
        if nmod < 1 or m < 1 or nt < 1 or nz < 1:
            raise ValueError("nmod, m, nt, nz must be >= 1")
        if width % 64 or c0 % 64 or c0 < nz + 2 * len(src_ix) + 1:
            raise ValueError("width and c0 must be multiples of 64, c0 >= nz + 2 ns + 1")
        self.dev = torch.device(device) if device is not None else torch.device("cuda")
        self.nmod, self.nz, self.nx, self.nt = nmod, nz, nx, nt
        self.ns, self.nr = len(src_ix), len(rec_ix)
        self.m, self.nimg = m, -(-nmod // m)
        self.amp, self.in_scale, self.in_shift = float(amp), float(in_scale), float(in_shift)
        self.c0, self.width = c0, width
        self.cout = -(-self.ns * nt // 256) * 256
        self.layers = layer_table(c0, width, self.cout)
        self.idx = {n: l for l, (n, _, _, _) in enumerate(self.layers)}
        hs = [nx]
        for _ in range(4):
            hs.append((hs[-1] + 1) // 2)
        self.half = hs                     # rows after 0..4 poolings of row pairs
        self.sizes = [hs[0], hs[2], hs[4]]
        self.shape = (nmod, nz, nx)
        i32 = dict(dtype=torch.int32, device=self.dev)
        self.rec_ix = torch.tensor([int(r) for r in rec_ix], **i32)
        col = np.full(nx, -1, np.int32)
        for r, x in enumerate(rec_ix):
            col[int(x)] = r
        self.col_rec = torch.tensor(col, **i32)
        self.G = torch.tensor(geometry_channels(nz, nx, src_ix, c0), device=self.dev)
        weights = weights if weights is not None else seeded_weights(c0, width, self.cout, seed)
        self._shapes = [((co, 3, ci), (co,)) for _, _, ci, co in self.layers]
        self.theta = torch.empty(sum(int(np.prod(s)) for sh in self._shapes for s in sh),
                                 dtype=torch.float32, device=self.dev)
        self.params = self.layer_views(self.theta)
        for (w, b), (wv, bv) in zip(weights, self.params):
            wv.copy_(torch.as_tensor(np.asarray(w, np.float32)))
            bv.copy_(torch.as_tensor(np.asarray(b, np.float32)))
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        self.W = [torch.empty((co, 3, 3, ci), **bf) for _, _, ci, co in self.layers]
        self.WT = [torch.empty((ci, 3, 3, co), **bf) for _, _, ci, co in self.layers]
        self.refresh()

        def act(k, c, dtype=torch.bfloat16):
            return torch.empty((self.nimg, self.sizes[k], m, c), dtype=dtype, device=self.dev)

        def half(j, c):     # a map after j poolings of row pairs
            return torch.empty((self.nimg, hs[j], m, c), dtype=torch.bfloat16, device=self.dev)

        w = width
        self.H = {j: half(j, w) for j in (1, 3)}       # the odd (half-way) sizes, forward
        self.dH = {j: half(j, w) for j in (1, 3)}      # and backward
        self.X0 = act(0, c0)
        self.P = {n: act(k, co) for n, k, _, co in self.layers if n != "out"}
        self.A = {n: act(k, co) for n, k, _, co in self.layers if n != "out"}
        self.D = {1: act(1, w), 2: act(2, w)}          # pooled encoder outputs
        self.U = {1: act(1, w), 0: act(0, w)}          # upsampled decoder inputs
        self.S = {1: act(1, w), 0: act(0, w)}          # after the additive skips
        self.Y = act(0, self.cout, torch.float32)
        self.dY = act(0, self.cout)
        self.dP = {n: act(k, co) for n, k, _, co in self.layers if n != "out"}
        self.dIn = {n: act(k, ci) for n, k, ci, _ in self.layers if n != "enc0"}
        self.dPool = {1: act(1, w), 2: act(2, w)}      # d/d(an upsampling input)
        self.dUp = {0: act(0, w), 1: act(1, w)}        # d/d(a pooling input)
        self.dAcc = {0: act(0, w), 1: act(1, w)}       # encoder outputs: skip + pooling
        self.dX = act(0, c0, torch.float32)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.d = torch.empty((nmod, self.ns, self.nr, nt), **f32)
        self.g = torch.empty(self.shape, **f32)

    # ------------------------------------------------------------- parameters
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

    def refresh(self, stream=None):
        """bf16 weights (zero horizontal taps) and their transposes from theta."""
        for l, (w3, _) in enumerate(self.params):
            api.fwi_sur_weights_prep(w3, self.W[l], self.WT[l], stream)

    def weights(self):
        """[(W3, b)] as float32 numpy arrays (for saving or the oracle)."""
        return [(w.detach().cpu().numpy().copy(), b.detach().cpu().numpy().copy())
                for w, b in self.params]

    # ------------------------------------------------------------- forward
    def _conv(self, name, x, stream):
        l = self.idx[name]
        api.fwi_conv3x3_bf16(x, self.W[l], self.params[l][1], 0, self.P[name], stream=stream)
        api.fwi_silu_bf16(self.P[name], self.A[name], stream)
        return self.A[name]

    def output(self, v: torch.Tensor, stream=None) -> torch.Tensor:
        """Y of the models v [nmod][nz][nx] (m/s); keeps the activations."""
        api.fwi_sur_pack(v, self.G, self.X0, self.m, self.in_scale, self.in_shift, stream)
        a0 = self._conv("enc0", self.X0, stream)
        api.fwi_pool_h_bf16(a0, self.H[1], 0, stream)
        api.fwi_pool_h_bf16(self.H[1], self.D[1], 0, stream)
        a1 = self._conv("enc1", self.D[1], stream)
        api.fwi_pool_h_bf16(a1, self.H[3], 0, stream)
        api.fwi_pool_h_bf16(self.H[3], self.D[2], 0, stream)
        a2 = self._conv("enc2", self.D[2], stream)
        api.fwi_up_h_bf16(a2, self.H[3], 0, stream)
        api.fwi_up_h_bf16(self.H[3], self.U[1], 0, stream)
        b1 = self._conv("dec1", self.U[1], stream)
        api.fwi_add_bf16(b1, a1, self.S[1], stream)
        api.fwi_up_h_bf16(self.S[1], self.H[1], 0, stream)
        api.fwi_up_h_bf16(self.H[1], self.U[0], 0, stream)
        b0 = self._conv("dec0", self.U[0], stream)
        api.fwi_add_bf16(b0, a0, self.S[0], stream)
        l = self.idx["out"]
        api.fwi_conv3x3_bf16(self.S[0], self.W[l], self.params[l][1], 0, self.Y, stream=stream)
        return self.Y

    def forward(self, v: torch.Tensor, d: torch.Tensor | None = None, stream=None):
        """The surrogate's seismograms d [nmod][ns][nr][nt] of models v."""
        self.output(v, stream)
        d = self.d if d is None else d
        api.fwi_sur_traces(self.Y, d, self.m, self.amp, self.rec_ix, stream)
        return d

    # ------------------------------------------------------------- backward
    def _layer_back(self, name, d, src, grads, work, stage, dW9, stream, act=True, dst=None):
        """Through one layer from the gradient d at its output: SiLU', the
        parameter gradients (with ``grads``) and the gradient at its input
        (into ``dst`` or dIn[name]; none when dst is False)."""
        l = self.idx[name]
        dp = self.dP[name] if act else d
        if act:
            api.fwi_silu_grad_bf16(d, self.P[name], dp, stream)
        if grads is not None:
            dW3, db = grads[l]
            api.fwi_conv3x3_wgrad_tc(src, dp, dW9[l], stage, work, stream=stream)
            api.fwi_sur_wgrad_centre(dW9[l], dW3, stream)
            api.fwi_channel_sum(dp, db, work, stream)
        if dst is False:
            return None
        dst = self.dIn[name] if dst is None else dst
        api.fwi_conv3x3_bf16(dp, self.WT[l], None, 0, dst, stream=stream)
        return dst

    def backward_from_output(self, grads=None, work=None, stage=None, dW9=None,
                             need_input=True, stream=None):
        """J^T through the network from dY (the gradient at Y, bf16, in
        self.dY): the parameter gradients into ``grads`` and, with need_input,
        the fp32 gradient at the packed input into self.dX."""
        ds0 = self._layer_back("out", self.dY, self.S[0], grads, work, stage, dW9, stream,
                               act=False)
        du0 = self._layer_back("dec0", ds0, self.U[0], grads, work, stage, dW9, stream)
        api.fwi_pool_h_bf16(du0, self.dH[1], 1, stream)           # adjoint of upsampling
        api.fwi_pool_h_bf16(self.dH[1], self.dPool[1], 1, stream)
        ds1 = self.dPool[1]
        du1 = self._layer_back("dec1", ds1, self.U[1], grads, work, stage, dW9, stream)
        api.fwi_pool_h_bf16(du1, self.dH[3], 1, stream)
        api.fwi_pool_h_bf16(self.dH[3], self.dPool[2], 1, stream)
        dd2 = self._layer_back("enc2", self.dPool[2], self.D[2], grads, work, stage, dW9, stream)
        api.fwi_up_h_bf16(dd2, self.dH[3], 1, stream)             # adjoint of mean pooling
        api.fwi_up_h_bf16(self.dH[3], self.dUp[1], 1, stream)
        api.fwi_add_bf16(ds1, self.dUp[1], self.dAcc[1], stream)
        dd1 = self._layer_back("enc1", self.dAcc[1], self.D[1], grads, work, stage, dW9, stream)
        api.fwi_up_h_bf16(dd1, self.dH[1], 1, stream)
        api.fwi_up_h_bf16(self.dH[1], self.dUp[0], 1, stream)
        api.fwi_add_bf16(ds0, self.dUp[0], self.dAcc[0], stream)
        self._layer_back("enc0", self.dAcc[0], self.X0, grads, work, stage, dW9, stream,
                         dst=self.dX if need_input else False)

    def vjp(self, adj: torch.Tensor, scale: float = 1.0, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
        """scale (dd/dv)^T adj [nmod][nz][nx] at the v of the last forward()."""
        api.fwi_sur_output_grad(self.Y, adj, self.dY, self.m, self.amp, self.col_rec, scale,
                                stream)
        self.backward_from_output(stream=stream)
        out = self.g if out is None else out
        api.fwi_sur_unpack_grad(self.dX, out, self.m, self.in_scale, stream)
        return out

    # ------------------------------------------------------------- training buffers
    def work_floats(self) -> int:
        return max(4 * 9 * ci * co for _, _, ci, co in self.layers)

    def stage_bytes(self) -> int:
        return max(api.fwi_conv3x3_wgrad_tc_stage_bytes(self.nimg, self.sizes[k], self.m, ci, co)
                   for _, k, ci, co in self.layers)


class SurrogateTrainer:
    """Supervised training of a ForwardSurrogate on FD pairs (v, d) with Adam
    (FP32 master parameters, bf16 weights refreshed after each step): the loss
    mean (Y - Yt)^2, Yt = sign(d) log(1 + |d| / amp) at the receivers (0
    elsewhere).  The minibatch is the network's nmod models (a multiple of m)."""

    def __init__(self, net: ForwardSurrogate, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        if net.nmod % net.m:
            raise ValueError("training needs nmod a multiple of m (no empty image columns)")
        self.net, self.lr, self.beta1, self.beta2, self.eps_adam = net, lr, beta1, beta2, eps
        f32 = dict(dtype=torch.float32, device=net.dev)
        self.grad = torch.zeros_like(net.theta)
        self.m1 = torch.zeros_like(net.theta)
        self.m2 = torch.zeros_like(net.theta)
        self.grads = net.layer_views(self.grad)
        self.dW9 = [torch.empty((co, 3, 3, ci), **f32) for _, _, ci, co in net.layers]
        self.Yt = torch.empty_like(net.Y)
        self.loss = torch.empty((1,), **f32)
        self.work = torch.empty(net.work_floats(), **f32)
        self.stage = torch.empty(net.stage_bytes(), dtype=torch.uint8, device=net.dev)
        self.k = 0

    def gradients(self, v: torch.Tensor, d: torch.Tensor, stream=None) -> torch.Tensor:
        """The loss on pairs (v [nmod][nz][nx], d [nmod][ns][nr][nt]) and its
        gradient with respect to theta in ``grad``."""
        net = self.net
        net.output(v, stream)
        api.fwi_sur_target(d, self.Yt, net.m, net.amp, net.col_rec, stream)
        api.fwi_sur_loss(net.Y, self.Yt, self.loss, net.dY, self.work, stream)
        net.backward_from_output(self.grads, self.work, self.stage, self.dW9, need_input=False,
                                 stream=stream)
        return self.loss

    def step(self, v: torch.Tensor, d: torch.Tensor, stream=None) -> torch.Tensor:
        loss = self.gradients(v, d, stream)
        self.k += 1
        api.fwi_adam_step(self.net.theta, self.grad, self.m1, self.m2, self.k, self.lr,
                          self.beta1, self.beta2, self.eps_adam, stream)
        self.net.refresh(stream)
        return loss


class SurrogateGuidance:
    """The surrogate's W2 guidance potential on a plan of the same models:
    J and dJ/dv of Eq. final_objective evaluated on the network's data --
    fwi_w2_misfit on the surrogate seismograms, then the network's
    vector-Jacobian product of the adjoint source."""

    def __init__(self, net: ForwardSurrogate, plan: api.Plan, ctx):
        if tuple(plan.model_shape) != net.shape:
            raise ValueError("the plan and the surrogate must hold the same models")
        self.net, self.plan, self.ctx = net, plan, ctx

    def gradient(self, v_phys: torch.Tensor, stream=None, step: int = -1):
        d = self.net.forward(v_phys, stream=stream)
        J, _, adj = self.plan.w2_misfit(self.ctx, d, stream=stream)
        return J, self.net.vjp(adj, stream=stream)


def rel_error(g: torch.Tensor, g_ref: torch.Tensor, stream=None) -> torch.Tensor:
    """Per-model relative L2 error ||g - g_ref|| / ||g_ref|| [nmod] (fwi_rel_error:
    the FD check's measure)."""
    return api.fwi_rel_error(g.contiguous(), g_ref.contiguous(), stream=stream)


@dataclasses.dataclass
class GateRecord:
    step: int
    error: float          # the largest per-model relative L2 error of that check
    accepted: bool


class GatedSurrogate:
    """The surrogate with the FD solver as check and fallback: at the first
    step it is asked for and then every ``check_every`` steps, both gradients
    are computed and the surrogate's relative L2 error against FD (the largest
    over the batch's models) is recorded; above ``threshold`` the step uses
    FD and every later step does too; otherwise the check step uses the FD
    gradient it has and the steps until the next check use the surrogate."""

    def __init__(self, surrogate: SurrogateGuidance, threshold: float = 0.05,
                 check_every: int = 10, measure=rel_error):
        self.sur, self.threshold, self.check_every = surrogate, float(threshold), int(check_every)
        self.measure = measure          # per-model relative error (fwi_rel_error)
        self.plan, self.ctx = surrogate.plan, surrogate.ctx
        self.records: list[GateRecord] = []
        self.rejected = False
        self._since = None
        self.n_surrogate = self.n_fd = 0

    def gradient(self, v_phys: torch.Tensor, stream=None, step: int = -1):
        if self.rejected:
            self.n_fd += 1
            J, g, _ = self.plan.gradient(v_phys, self.ctx, stream=stream)
            return J, g
        if self._since is None or self._since >= self.check_every:
            J, g_fd, _ = self.plan.gradient(v_phys, self.ctx, stream=stream)
            g_fd = g_fd.clone()
            _, g_sur = self.sur.gradient(v_phys, stream=stream)
            err = float(self.measure(g_sur, g_fd).max())
            ok = err <= self.threshold
            self.records.append(GateRecord(step, err, ok))
            self.rejected = not ok
            self._since = 1
            self.n_fd += 1
            return J, g_fd
        self._since += 1
        self.n_surrogate += 1
        return self.sur.gradient(v_phys, stream=stream)


# ----------------------------------------------------------------- training data
def fd_pairs(plan: api.Plan, models, stream=None):
    """(v [N][nz][nx], d [N][ns][nr][nt]) on the plan's device: the FD
    seismograms (fwi_forward, no record) of N models (host array, m/s),
    plan.batch at a time; N must be a multiple of the plan's batch."""
    B = plan.model_shape[0]
    if torch.is_tensor(models):
        v = models.to(device=plan.device, dtype=torch.float32).contiguous()
    else:
        v = torch.tensor(np.asarray(models, np.float32), device=plan.device)
    N = v.shape[0]
    if N % B:
        raise ValueError(f"{N} models are not a multiple of the plan's batch {B}")
    d = torch.empty((N,) + tuple(plan.data_shape[1:]), dtype=torch.float32, device=plan.device)
    for k in range(0, N, B):
        dk, _ = plan.forward(v[k:k + B], store=False, stream=stream)
        d[k:k + B].copy_(dk)
    return v, d


def trace_amplitude(d: torch.Tensor, k: float = 100.0) -> float:
    """amp = max |d| / k: the trace map's scale, so that y = sign(d) log(1 + |d|/amp)
    compresses the largest amplitude to log(1 + k) (k = 100 mirrors the W2
    weighting's k of Eq. omega_def)."""
    return float(d.abs().max()) / k


def train(trainer: SurrogateTrainer, v: torch.Tensor, d: torch.Tensor, steps: int,
          stream=None, log_every: int = 0):
    """``steps`` Adam steps over the dataset in order, one minibatch of the
    network's nmod consecutive pairs each (the dataset wraps around); returns
    [(step, loss)] read back every ``log_every`` steps (0: only the last)."""
    B, N = trainer.net.nmod, v.shape[0]
    if N < B:
        raise ValueError("fewer pairs than one minibatch")
    nb = N // B
    out = []
    loss = None
    for k in range(steps):
        o = (k % nb) * B
        loss = trainer.step(v[o:o + B], d[o:o + B], stream)
        if log_every and (k + 1) % log_every == 0:
            out.append((k + 1, float(loss.item())))
    if loss is not None and (not out or out[-1][0] != steps):
        out.append((steps, float(loss.item())))
    return out


def copy_weights(dst: ForwardSurrogate, src: ForwardSurrogate):
    """Give dst (another batch size) the parameters of src."""
    if dst.theta.numel() != src.theta.numel():
        raise ValueError("the networks differ in architecture")
    dst.theta.copy_(src.theta)
    dst.amp = src.amp
    dst.refresh()


def early_clean_estimates(models: torch.Tensor, prior, betas: Sequence[float], i_lo: int,
                          i_hi: int, chunk: int, seed: int = 0,
                          space: api.DiffusionSpace = api.DiffusionSpace(),
                          sigma_mode: int = api.SIGMA_POSTERIOR) -> torch.Tensor:
    """The physical models a reverse diffusion hands its guidance in steps
    i_lo..i_hi: each chunk of ``chunk`` models [N][nz][nx] (m/s, device) is
    noised to a step i drawn uniformly from that range (fwi_dsm_noisy: x_i =
    sqrt(abar_i) x_0 + sqrt(1 - abar_i) z, x_0 = (v - shift) / unit) and
    mapped to its clamped clean estimate under the Gaussian prior
    (fwi_ddpm_proposal's v_phys) -- the inputs the surrogate is queried on in
    the early, high-noise steps, which it is trained on."""
    N, nz, nx = models.shape
    if N % chunk:
        raise ValueError("the number of models must be a multiple of chunk")
    dev = models.device
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev).manual_seed(seed)
    x0 = ((models - space.shift) / space.unit).contiguous()
    out = torch.empty_like(models)
    z = torch.empty((chunk, nz, nx), dtype=torch.float32, device=dev)
    xt = torch.empty_like(z)
    v0, vp = torch.empty_like(z), torch.empty_like(z)
    zero = torch.zeros_like(z)
    for k in range(0, N, chunk):
        i = int(rng.integers(i_lo, i_hi + 1))
        st = api.fwi_ddpm_coefficients(list(betas), i, sigma_mode)
        z.normal_(generator=gen)
        api.fwi_dsm_noisy(x0[k:k + chunk], z, st.abar, xt)
        api.fwi_ddpm_proposal(chunk, nz * nx, st, space, xt, None, prior.mu, prior.tau2, zero,
                              v0, vp, out[k:k + chunk])
    return out
