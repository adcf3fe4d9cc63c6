"""FP64 oracle of the U-Net noise-prediction score network (the score model of
Sec. 6 is a U-Net; the architecture is a reading): four levels of widths
c_0..c_3; per encoder level two 3x3 convolution + SiLU layers, 2 x 2 mean
pooling between levels; per decoder level (2, 1, 0) nearest upsampling of the
deeper output to the level's size, a convolution + SiLU, the encoder's output
of the level added, a second convolution + SiLU; a last linear convolution
whose channel 0 is eps.  The input enters as channel 0 of c_0 channels; the
step i enters every layer's bias as b + E phi(i).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
numpy in float64, convolutions from ``oracle/conv.py``.  With round_bf16 the
values a bf16 network stores are rounded to bfloat16 at the same points (the
input channel, pre-activations, activations, pooled, upsampled and summed
maps, the output gradient and every gradient between layers).
"""
from __future__ import annotations

import numpy as np

from . import conv as C
from . import score_net as N
from . import score_train as T


def pool2(x, mode=0):
    """[n][h][w][c] -> [n][(h+1)/2][(w+1)/2][c]: the mean (mode 0) or the sum
    (mode 1) of each 2 x 2 block's cells inside the image."""
    x = np.asarray(x, np.float64)
    n, h, w, c = x.shape
    hc, wc = (h + 1) // 2, (w + 1) // 2
    y = np.zeros((n, hc, wc, c))
    for I in range(hc):
        for J in range(wc):
            blk = x[:, 2 * I:2 * I + 2, 2 * J:2 * J + 2, :]
            s = blk.sum(axis=(1, 2))
            y[:, I, J, :] = s / (blk.shape[1] * blk.shape[2]) if mode == 0 else s
    return y


def up2(x, ho, wo, mode=0):
    """[n][(ho+1)/2][(wo+1)/2][c] -> [n][ho][wo][c]: y[i][j] = x[i/2][j/2]
    (mode 0), divided by the cells of block (i/2, j/2) inside ho x wo (mode 1)."""
    x = np.asarray(x, np.float64)
    y = np.zeros((x.shape[0], ho, wo, x.shape[3]))
    for i in range(ho):
        for j in range(wo):
            cnt = (min(2 * (i // 2) + 2, ho) - 2 * (i // 2)) * (min(2 * (j // 2) + 2, wo) - 2 * (j // 2))
            y[:, i, j, :] = x[:, i // 2, j // 2, :] / (cnt if mode == 1 else 1)
    return y


def layers(widths):
    c = widths
    out = []
    for k in range(4):
        out += [(f"enc{k}a", c[0] if k == 0 else c[k - 1], c[k]), (f"enc{k}b", c[k], c[k])]
    for k in (2, 1, 0):
        out += [(f"dec{k}u", c[k + 1], c[k]), (f"dec{k}c", c[k], c[k])]
    out.append(("out", c[0], c[0]))
    return out


class UNet:
    """weights: [(W [cout][3][3][cin], b, E)] in the order of ``layers``."""

    def __init__(self, weights, widths, round_bf16: bool = True):
        self.r = N.bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
        self.names = [n for n, _, _ in layers(widths)]
        self.W = {n: self.r(w) for n, (w, _, _) in zip(self.names, weights)}
        self.b = {n: np.asarray(b, np.float64) for n, (_, b, _) in zip(self.names, weights)}
        self.E = {n: np.asarray(e, np.float64) for n, (_, _, e) in zip(self.names, weights)}
        self.c = widths
        self.f32 = round_bf16

    def bias(self, name, i):
        b = self.b[name] + self.E[name] @ N.time_features(i, self.E[name].shape[1])
        return b.astype(np.float32).astype(np.float64) if self.f32 else b

    def _layer(self, name, x, i):
        p = self.r(C.conv3x3(x, self.W[name], self.bias(name, i)))
        self.P[name], self.In[name] = p, x
        return self.r(N.silu(p))

    def eps(self, x, i):
        r = self.r
        x = np.asarray(x, np.float64)
        self.P, self.In, self.sizes = {}, {}, [x.shape[1:3]]
        h = np.zeros(x.shape + (self.c[0],))
        h[..., 0] = r(x)
        enc = {}
        for k in range(4):
            if k > 0:
                h = r(pool2(h, 0))
                self.sizes.append(h.shape[1:3])
            h = self._layer(f"enc{k}a", h, i)
            h = enc[k] = self._layer(f"enc{k}b", h, i)
        for k in (2, 1, 0):
            ho, wo = self.sizes[k]
            u = up2(h, ho, wo, 0)
            a = self._layer(f"dec{k}u", u, i)
            s = r(a + enc[k])
            h = self._layer(f"dec{k}c", s, i)
        self.In["out"] = h
        return C.conv3x3(h, self.W["out"], self.bias("out", i))[..., 0]

    def _back(self, name, d, act=True):
        """(dP, gradient at the layer's input) from the gradient d at its output."""
        r = self.r
        dp = r(r(d) * N.silu_grad(self.P[name])) if act else d
        wt = np.flip(self.W[name], axis=(1, 2)).transpose(3, 1, 2, 0)
        self.dPs[name] = dp
        return dp, C.conv3x3(dp, wt)

    def backward(self, g, scale=1.0):
        """Fills dPs (each layer's output-side gradient) and returns J^T (scale g)."""
        r = self.r
        self.dPs = {}
        g = np.asarray(g, np.float64)
        d = np.zeros(g.shape + (self.c[0],))
        d[..., 0] = r(scale * g)
        _, d = self._back("out", d, act=False)
        d = r(d)
        dskip = {}
        for k in (0, 1, 2):
            _, ds = self._back(f"dec{k}c", d)
            ds = dskip[k] = r(ds)
            _, du = self._back(f"dec{k}u", ds)
            d = r(pool2(r(du), 1))
        for k in (3, 2, 1, 0):
            if k < 3:
                d = r(d + dskip[k])
            _, da = self._back(f"enc{k}b", d)
            _, dd = self._back(f"enc{k}a", r(da))
            if k > 0:
                ho, wo = self.sizes[k - 1]
                d = r(up2(r(dd), ho, wo, 1))
        return dd[..., 0]

    def param_grads(self, i):
        """[(dW, db, dE)] in layer order after backward()."""
        phi = N.time_features(i, self.E["out"].shape[1])
        out = []
        for name in self.names:
            dp = self.dPs[name]
            db = T.channel_sum(dp)
            out.append((T.conv3x3_wgrad(self.In[name], dp), db, np.outer(db, phi)))
        return out


def dsm_gradients(weights, widths, x0, z, abar, t, round_bf16: bool = True):
    """(loss, [(dW, db, dE)]) of one minibatch at step t (Eq. L2_rewrite with
    kappa = 1 - abar, as in ``oracle/score_train.py``)."""
    net = UNet(weights, widths, round_bf16)
    eps = net.eps(T.noisy(x0, z, abar), t)
    loss, g = T.dsm_loss(eps, z)
    net.backward(g)
    return loss, net.param_grads(t)
