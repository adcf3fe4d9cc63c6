"""FP64 oracle of denoising-score-matching training (Sec. 3.4, Eq. L2_rewrite)
for the convolutional noise-prediction score model of ``oracle/score_net.py``.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
numpy in float64, each function the definition written out:

  noisy:       x_t = sqrt(abar) x_0 + sqrt(1 - abar) z, a draw of the VP
               transition q_t(. | x_0) (Eq. vp_transition)
  dsm_loss:    with s = -eps / sqrt(1 - abar) and the conditional score
               -(x_t - sqrt(abar) x_0) / (1 - abar) = -z / sqrt(1 - abar),
               the integrand of Eq. L2_rewrite weighted by kappa = 1 - abar is
               ||eps - z||^2; the loss is its mean over the entries, and its
               gradient 2 (eps - z) / n
  conv3x3_wgrad: dW[co][ky][kx][ci] = sum_{b,p} dP[b][p][co] x[b][p + (ky-1, kx-1)][ci],
               the gradient of W -> <conv3x3(x, W), dP>
  channel_sum: db[c] = sum_{b,p} dP[b][p][c]
  adam:        Adam (Kingma and Ba, 2015) with bias-corrected moments
  time_bias:   the per-step biases b + E phi(i)
  dsm_gradients: the loss of one minibatch at one step t and its gradient
               with respect to every (W, b, E), by the chain rule through the
               network of ``oracle/score_net.py`` (bf16 storage points as there)
  regression_gradients: the same for the supervised loss mean (eps(x) - y)^2
"""
from __future__ import annotations

import numpy as np

from . import conv as C
from . import score_net as N


def noisy(x0, z, abar):
    return np.sqrt(abar) * np.asarray(x0, np.float64) + np.sqrt(1.0 - abar) * np.asarray(z, np.float64)


def dsm_loss(eps, z):
    """(mean (eps - z)^2, d/d eps)."""
    d = np.asarray(eps, np.float64) - np.asarray(z, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def conv3x3_wgrad(x, dp):
    """x [n][h][w][cin], dP [n][h][w][cout] -> dW [cout][3][3][cin]."""
    x = np.asarray(x, np.float64)
    dp = np.asarray(dp, np.float64)
    n, h, w, cin = x.shape
    cout = dp.shape[-1]
    xp = np.zeros((n, h + 2, w + 2, cin))
    xp[:, 1:h + 1, 1:w + 1] = x
    dw = np.zeros((cout, 3, 3, cin))
    P = dp.reshape(-1, cout)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = P.T @ xp[:, ky:ky + h, kx:kx + w, :].reshape(-1, cin)
    return dw


def channel_sum(dp):
    dp = np.asarray(dp, np.float64)
    return dp.reshape(-1, dp.shape[-1]).sum(axis=0)


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number ``step`` >= 1: returns (p, m, v)."""
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return np.asarray(p, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def time_bias(b, E, phi):
    """b [C], E [C][dim], phi [..][dim] -> [..][C]."""
    return np.asarray(b, np.float64) + np.asarray(phi, np.float64) @ np.asarray(E, np.float64).T


def dsm_gradients(weights, x0, z, abar, t, round_bf16: bool = True):
    """(loss, [(dW, db, dE)] per layer) of one minibatch x0, z [B][nz][nx] at
    step t."""
    return _gradients(weights, noisy(x0, z, abar), z, t, round_bf16)


def regression_gradients(weights, x, y, i=0, in_scale=1.0, round_bf16: bool = True):
    """(loss, [(dW, db, dE)]) of the supervised regression mean (eps(in_scale x, i) - y)^2
    (a network surrogate trained on pairs)."""
    return _gradients(weights, in_scale * np.asarray(x, np.float64), y, i, round_bf16)


def _gradients(weights, xt, z, t, round_bf16):
    net = N.ConvScore(weights, round_bf16=round_bf16)
    r = net.r
    eps = net.eps(xt, t)
    loss, g = dsm_loss(eps, z)
    L = len(net.W)
    inputs = [np.zeros(xt.shape + (net.Cn,))]
    inputs[0][..., 0] = r(xt)
    for l in range(L - 1):
        inputs.append(r(N.silu(net.P[l])))
    phi = N.time_features(t, net.E[0].shape[1])
    d = np.zeros(xt.shape + (net.Cn,))
    d[..., 0] = r(g)
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        dw = conv3x3_wgrad(inputs[l], d)
        db = channel_sum(d)
        grads[l] = (dw, db, np.outer(db, phi))
        if l > 0:
            wt = np.flip(net.W[l], axis=(1, 2)).transpose(3, 1, 2, 0)
            d = r(r(C.conv3x3(d, wt)) * N.silu_grad(net.P[l - 1]))
    return loss, grads
