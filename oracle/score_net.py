"""FP64 oracle of the convolutional score model (noise prediction, Sec. 3.4):
s(x, i) = -eps(x) / sqrt(1 - abar_i), eps = L 3x3 convolution layers with
SiLU between them, the state entering as channel 0 and eps read from
channel 0 of the last layer, and its vector-Jacobian product.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
numpy in float64, the convolution from ``oracle/conv.py``.  With
``bf16=True`` the values a bf16 network stores (the input channel, the
pre-activations and activations, the scaled output gradient and the
gradients between layers) are rounded to bfloat16 (round to nearest even)
at the same points; with ``bf16=False`` nothing is rounded.
"""
from __future__ import annotations

import numpy as np

from . import conv as C


def bf16(a):
    """Round to bfloat16 (nearest even), returned as float64."""
    x = np.asarray(a, dtype=np.float64).astype(np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(p):
    return p / (1.0 + np.exp(-p))


def silu_grad(p):
    sg = 1.0 / (1.0 + np.exp(-p))
    return sg * (1.0 + p * (1.0 - sg))


def time_features(i: int, dim: int = 16):
    """[sin(i w_k), cos(i w_k)], w_k = 10000^(-k / (dim/2)): the step's embedding."""
    k = np.arange(dim // 2, dtype=np.float64)
    w = 10000.0 ** (-k / (dim // 2))
    return np.concatenate([np.sin(i * w), np.cos(i * w)])


class ConvScore:
    """weights: [(W [C][3][3][C], b [C], E [C][dim])]; layer l's bias at step i
    is b_l + E_l phi(i), rounded to float32 as the kernels receive it."""

    def __init__(self, weights, round_bf16: bool = True):
        self.r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
        self.W = [self.r(w) for w, _, _ in weights]
        self.b = [np.asarray(b, np.float64) for _, b, _ in weights]
        self.E = [np.asarray(e, np.float64) for _, _, e in weights]
        self.f32 = round_bf16
        self.Cn = self.W[0].shape[0]

    def bias(self, l, i):
        b = self.b[l] + self.E[l] @ time_features(i, self.E[l].shape[1])
        return b.astype(np.float32).astype(np.float64) if self.f32 else b

    def eps(self, x, i=0):
        """eps(x, i) for x [B][nz][nx]; keeps the pre-activations for vjp."""
        x = np.asarray(x, np.float64)
        h = np.zeros(x.shape + (self.Cn,))
        h[..., 0] = self.r(x)
        self.P = []
        L = len(self.W)
        for l in range(L):
            p = C.conv3x3(h, self.W[l], self.bias(l, i))
            if l < L - 1:
                p = self.r(p)
                self.P.append(p)
                h = self.r(silu(p))
            else:
                y = p
        return y[..., 0]

    def eps_vjp(self, g, scale=1.0):
        """scale J_eps^T g at the x of the last eps() call."""
        g = np.asarray(g, np.float64)
        d = np.zeros(g.shape + (self.Cn,))
        d[..., 0] = self.r(scale * g)
        for l in range(len(self.W) - 1, -1, -1):
            # the adjoint of the zero-padded convolution: taps flipped, channels swapped
            wt = np.flip(self.W[l], axis=(1, 2)).transpose(3, 1, 2, 0)
            d = C.conv3x3(d, wt)
            if l > 0:
                d = self.r(self.r(d) * silu_grad(self.P[l - 1]))
        return d[..., 0]

    def score(self, x, abar, i=0):
        return -self.eps(x, i) / np.sqrt(1.0 - abar)

    def score_vjp(self, g, abar):
        return self.eps_vjp(g, -1.0 / np.sqrt(1.0 - abar))
