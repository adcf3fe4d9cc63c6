"""FP64 oracle of the learned forward surrogate: a convolutional
encoder-decoder mapping a velocity model to the seismograms of the FD solver
(the surrogate route to cheaper guidance that Sec. 7 proposes, used in the
early reverse steps of Algorithm 2, Sec. 5.2), its vector-Jacobian product
(the surrogate's W2 guidance gradient is that product applied to the W2
adjoint source of Eq. final_objective) and the gradients of its supervised
training loss.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
numpy in float64; the 3x3 convolution from ``oracle/conv.py``.

The network, per model b (the architecture is a reading; the paper gives none):
  input   X0 [nx][1][C0]: column x of the model is pixel x of a one-pixel-wide
          image; channel z < nz holds in_scale v[z][x] + in_shift, the channels
          above hold fixed geometry features G[x][c] (per shot s the offset
          (x - src_ix[s]) / nx and its magnitude, then a constant 1)
  layers  six convolutions with three taps along the image (pixel x couples
          to x - 1, x, x + 1; weights W3 [cout][3][cin], bias b):
            enc0 (level 0) -> mean pooling by 4 -> enc1 (level 1) -> pooling ->
            enc2 (level 2) -> nearest upsampling by 4 -> dec1 (level 1) + enc1's
            output -> upsampling -> dec0 (level 0) + enc0's output -> out
          SiLU after every layer but ``out``; pooling by 4 is two poolings of
          row pairs (ceil(h / 2) rows each), upsampling by 4 two nearest
          doublings back through the same sizes, so level 2 of a 70-column
          model has 5 pixels and the bottleneck sees the whole model
  output  y = Y[x][s nt + t] of the linear ``out`` layer, and the trace of
          receiver r (at column rec_ix[r]) is d[s][r][t] = amp sign(y) (e^|y| - 1),
          the inverse of the compressive map y = sign(d) log(1 + |d| / amp)
          (which gives weak arrivals weight in the fit, as the W2 weighting
          omega of Eq. omega_def does in the misfit)
The GPU keeps several models side by side in one image (w = models per image)
with the taps of the horizontal neighbours fixed at zero, which computes
exactly this per-model network.  With round_bf16 the values the bf16 network
stores are rounded to bfloat16 at the same points as on the GPU (input,
pre-activations, activations, pooled and summed maps, the output gradient and
every gradient between layers); the last layer's output and the input
gradient are float.
"""
from __future__ import annotations

import numpy as np

from . import conv as C
from . import score_net as N
from . import score_train as T

LAYERS = ("enc0", "enc1", "enc2", "dec1", "dec0", "out")
LEVEL = {"enc0": 0, "enc1": 1, "enc2": 2, "dec1": 1, "dec0": 0, "out": 0}


def layer_table(c0: int, width: int, cout: int):
    """[(name, level, cin, cout)] of the six convolutions, in parameter order."""
    return [("enc0", 0, c0, width), ("enc1", 1, width, width), ("enc2", 2, width, width),
            ("dec1", 1, width, width), ("dec0", 0, width, width), ("out", 0, width, cout)]


def geometry_channels(nz: int, nx: int, src_ix, c0: int):
    """G [nx][c0]: zero below channel nz; per shot s the offset (x - src_ix[s]) / nx
    (channel nz + 2 s) and its magnitude (nz + 2 s + 1); then 1 (nz + 2 ns)."""
    ns = len(src_ix)
    if nz + 2 * ns + 1 > c0:
        raise ValueError("c0 too small for nz + 2 ns + 1 input channels")
    G = np.zeros((nx, c0))
    x = np.arange(nx, dtype=np.float64)
    for s, sx in enumerate(src_ix):
        G[:, nz + 2 * s] = (x - sx) / nx
        G[:, nz + 2 * s + 1] = np.abs(x - sx) / nx
    G[:, nz + 2 * ns] = 1.0
    return G


def expand_taps(w3):
    """W3 [cout][3][cin] -> the 3 x 3 convolution weights [cout][3][3][cin]
    whose horizontal taps (kx = 0, 2) are zero."""
    w3 = np.asarray(w3, np.float64)
    w = np.zeros((w3.shape[0], 3, 3, w3.shape[2]))
    w[:, :, 1, :] = w3
    return w


def pool_h(x, mode=0):
    """[n][h][w][c] -> [n][(h+1)/2][w][c]: mean (mode 0) or sum (mode 1) of
    the rows 2I, 2I + 1 inside the image."""
    x = np.asarray(x, np.float64)
    n, h, w, c = x.shape
    y = np.zeros((n, (h + 1) // 2, w, c))
    for I in range(y.shape[1]):
        blk = x[:, 2 * I:2 * I + 2]
        y[:, I] = blk.sum(axis=1) / (blk.shape[1] if mode == 0 else 1)
    return y


def up_h(x, ho, mode=0):
    """[n][(ho+1)/2][w][c] -> [n][ho][w][c]: y[i] = x[i/2] (mode 0), divided by
    the rows of block i/2 inside ho (mode 1; the adjoint of pool_h mode 0)."""
    x = np.asarray(x, np.float64)
    y = np.zeros((x.shape[0], ho) + x.shape[2:])
    for i in range(ho):
        cnt = min(2 * (i // 2) + 2, ho) - 2 * (i // 2)
        y[:, i] = x[:, i // 2] / (cnt if mode == 1 else 1)
    return y


def slog(d, amp):
    """The compressive map of the traces: sign(d) log(1 + |d| / amp)."""
    d = np.asarray(d, np.float64)
    return np.sign(d) * np.log1p(np.abs(d) / amp)


def slog_inv(y, amp):
    """amp sign(y) (e^|y| - 1), the inverse of slog."""
    y = np.asarray(y, np.float64)
    return amp * np.sign(y) * np.expm1(np.abs(y))


def seeded_weights(c0: int, width: int, cout: int, seed: int = 0):
    """[(W3 [cout][3][cin], b [cout])] float32: W3 of variance 1/(3 cin) (the
    SiLU layers) or 1/(3 cin) / 16 (the output layer, whose fit starts small),
    b zero."""
    rng = np.random.default_rng(seed)
    out = []
    for name, _, ci, co in layer_table(c0, width, cout):
        w = rng.standard_normal((co, 3, ci)) / np.sqrt(3 * ci)
        if name == "out":
            w /= 4.0
        out.append((w.astype(np.float32), np.zeros(co, np.float32)))
    return out


class Surrogate:
    """weights: [(W3 [cout][3][cin], b [cout])] in the order of LAYERS.
    rec_ix: the receivers' columns (distinct); src_ix: the shots' columns."""

    def __init__(self, weights, nz, nx, nt, src_ix, rec_ix, amp, c0, in_scale=1.0,
                 in_shift=0.0, round_bf16: bool = True):
        self.r = N.bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
        self.W = {n: self.r(expand_taps(w)) for n, (w, _) in zip(LAYERS, weights)}
        f32 = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if round_bf16 else \
            (lambda a: np.asarray(a, np.float64))
        self.b = {n: f32(b) for n, (_, b) in zip(LAYERS, weights)}
        self.nz, self.nx, self.nt = nz, nx, nt
        self.src_ix, self.rec_ix = list(src_ix), list(rec_ix)
        self.ns, self.nr = len(self.src_ix), len(self.rec_ix)
        self.amp, self.c0 = float(amp), c0
        self.in_scale, self.in_shift = float(in_scale), float(in_shift)
        self.G = geometry_channels(nz, nx, self.src_ix, c0)
        h = [nx]
        for _ in range(4):
            h.append((h[-1] + 1) // 2)
        self.half = h              # rows after 0..4 poolings of row pairs
        self.sizes = [h[0], h[2], h[4]]

    def pack(self, v):
        """X0 [B][nx][1][c0] of models v [B][nz][nx] (before rounding)."""
        v = np.asarray(v, np.float64)
        X = np.repeat(self.G[None, :, None, :], v.shape[0], axis=0)
        X[:, :, 0, :self.nz] = self.in_scale * v.transpose(0, 2, 1) + self.in_shift
        return X

    def _layer(self, name, x, act=True):
        p = C.conv3x3(x, self.W[name], self.b[name])
        self.In[name] = x
        if not act:
            return p
        p = self.r(p)
        self.P[name] = p
        return self.r(N.silu(p))

    def output(self, v):
        """Y [B][nx][1][cout] of the last layer (float, before the trace map)."""
        r = self.r
        self.P, self.In = {}, {}
        h = self.half
        x0 = r(self.pack(v))
        a0 = self.A0 = self._layer("enc0", x0)
        a1 = self.A1 = self._layer("enc1", r(pool_h(r(pool_h(a0, 0)), 0)))
        a2 = self._layer("enc2", r(pool_h(r(pool_h(a1, 0)), 0)))
        b1 = self._layer("dec1", up_h(up_h(a2, h[3], 0), h[2], 0))
        s1 = r(b1 + a1)
        b0 = self._layer("dec0", up_h(up_h(s1, h[1], 0), h[0], 0))
        s0 = r(b0 + a0)
        self.Y = self._layer("out", s0, act=False)
        return self.Y

    def traces(self, Y=None):
        """d [B][ns][nr][nt] from Y (default: the last output)."""
        Y = self.Y if Y is None else Y
        B = Y.shape[0]
        d = np.zeros((B, self.ns, self.nr, self.nt))
        for s in range(self.ns):
            for r, x in enumerate(self.rec_ix):
                d[:, s, r, :] = slog_inv(Y[:, x, 0, s * self.nt:(s + 1) * self.nt], self.amp)
        return d

    def forward(self, v):
        self.output(v)
        return self.traces()

    def target(self, d):
        """Yt [B][nx][1][cout]: slog of the traces at the receivers' columns, 0
        elsewhere (the regression target of Y)."""
        d = np.asarray(d, np.float64)
        Yt = np.zeros((d.shape[0], self.nx, 1, self.W["out"].shape[0]))
        for s in range(self.ns):
            for r, x in enumerate(self.rec_ix):
                Yt[:, x, 0, s * self.nt:(s + 1) * self.nt] = slog(d[:, s, r, :], self.amp)
        return Yt

    def _back(self, name, d, act=True):
        """(dP, gradient at the layer's input) from the gradient d at its output."""
        r = self.r
        dp = r(r(d) * N.silu_grad(self.P[name])) if act else d
        self.dPs[name] = dp
        wt = np.flip(self.W[name], axis=(1, 2)).transpose(3, 1, 2, 0)
        return C.conv3x3(dp, wt)

    def backward_from_output(self, dY):
        """J^T through the network from the gradient dY at Y (already in the
        stored precision); returns the gradient at v [B][nz][nx]."""
        r = self.r
        self.dPs = {}
        h = self.half
        ds0 = r(self._back("out", dY, act=False))
        du0 = r(self._back("dec0", ds0))
        ds1 = r(pool_h(r(pool_h(du0, 1)), 1))
        du1 = r(self._back("dec1", ds1))
        da2 = r(pool_h(r(pool_h(du1, 1)), 1))
        dd2 = r(self._back("enc2", da2))
        da1 = r(ds1 + r(up_h(r(up_h(dd2, h[3], 1)), h[2], 1)))
        dd1 = r(self._back("enc1", da1))
        da0 = r(ds0 + r(up_h(r(up_h(dd1, h[1], 1)), h[0], 1)))
        dx0 = self._back("enc0", da0)
        return self.in_scale * dx0[:, :, 0, :self.nz].transpose(0, 2, 1)

    def output_grad(self, adj, scale=1.0):
        """dY [B][nx][1][cout] of an adjoint source adj [B][ns][nr][nt] (the
        trace map's derivative amp e^|y| applied), rounded to bf16."""
        adj = np.asarray(adj, np.float64)
        dY = np.zeros_like(self.Y)
        for s in range(self.ns):
            for r, x in enumerate(self.rec_ix):
                y = self.Y[:, x, 0, s * self.nt:(s + 1) * self.nt]
                dY[:, x, 0, s * self.nt:(s + 1) * self.nt] = \
                    scale * adj[:, s, r, :] * self.amp * np.exp(np.abs(y))
        return self.r(dY)

    def vjp(self, adj, scale=1.0):
        """scale (dd/dv)^T adj at the v of the last forward()."""
        return self.backward_from_output(self.output_grad(adj, scale))

    def param_grads(self):
        """[(dW3, db)] in layer order after a backward pass: the centre column of
        the 3 x 3 weight gradient (the only taps the network has)."""
        out = []
        for name in LAYERS:
            dp = self.dPs[name]
            out.append((T.conv3x3_wgrad(self.In[name], dp)[:, :, 1, :], T.channel_sum(dp)))
        return out


def regression_loss(Y, Yt):
    """(mean (Y - Yt)^2 over every entry, its gradient 2 (Y - Yt) / n)."""
    d = np.asarray(Y, np.float64) - np.asarray(Yt, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def training_gradients(net: Surrogate, v, d):
    """(loss, [(dW3, db)]) of the supervised loss on pairs (v, d): the network's
    output Y against slog(d) at the receivers (0 elsewhere)."""
    Y = net.output(v)
    loss, g = regression_loss(Y, net.target(d))
    net.backward_from_output(net.r(g))
    return loss, net.param_grads()
