"""FP64 oracle of the 3x3 convolution (stride 1, zero padding 1) that the
tensor-core kernel computes, the dense contraction of a convolutional score
model or surrogate for the guidance of Algorithms 1-2 (a U-Net in Sec. 6; the
surrogate idea in Sec. 7):

    y[b][p][co] = act(bias[co] + sum_{ky,kx,ci} x[b][p + (ky-1, kx-1)][ci] w[co][ky][kx][ci])

with x read as 0 outside the image and act the identity or SiLU v/(1 + e^-v).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.  numpy in float64: the definition
written out, one tap at a time, each tap a matrix product over channels.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, bias=None, act: int = 0):
    """x [n][h][w][cin], w [cout][3][3][cin], bias [cout] or None -> y [n][h][w][cout]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, h, wd, cin = x.shape
    cout = w.shape[0]
    xp = np.zeros((n, h + 2, wd + 2, cin))
    xp[:, 1:h + 1, 1:wd + 1, :] = x
    y = np.zeros((n, h, wd, cout))
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + h, kx:kx + wd, :] @ w[:, ky, kx, :].T
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)
    if act == 1:
        y = y / (1.0 + np.exp(-y))
    return y


def abs_sum(x, w):
    """sum_{ky,kx,ci} |x[p + tap][ci]| |w[co][tap][ci]| per output: the scale
    of the rounding error of any summation order of the products."""
    return conv3x3(np.abs(np.asarray(x, np.float64)), np.abs(np.asarray(w, np.float64)))


def conv3x3_at(x, w, bias, act, pixels, channels):
    """y at the listed (b, iy, ix) pixels and output channels only (for
    sampled checks of large launches): [len(pixels)][len(channels)]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)[list(channels)]
    n, h, wd, cin = x.shape
    out = np.zeros((len(pixels), len(channels)))
    for k, (b, iy, ix) in enumerate(pixels):
        acc = np.zeros(len(channels))
        for ky in range(3):
            for kx in range(3):
                yy, xx = iy + ky - 1, ix + kx - 1
                if 0 <= yy < h and 0 <= xx < wd:
                    acc += w[:, ky, kx, :] @ x[b, yy, xx, :]
        if bias is not None:
            acc += np.asarray(bias, dtype=np.float64)[list(channels)]
        out[k] = acc / (1.0 + np.exp(-acc)) if act == 1 else acc
    return out
