"""Pins of the denoising-score-matching oracle (``oracle/score_train.py``),
CPU only: the weight gradient and the channel sum against the linear
functionals they differentiate (through ``oracle/conv.py``), the whole
minibatch gradient against central differences of the unrounded loss, the
DSM loss against the conditional score of Eq. L2_rewrite written from the
Gaussian transition, and Adam against its closed forms."""
import numpy as np

from oracle import conv as C
from oracle import score_net as N
from oracle import score_train as T


def _weights(seed=0, c=4, layers=3):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((c, 3, 3, c)) / np.sqrt(9 * c), 0.1 * rng.standard_normal(c),
             0.1 * rng.standard_normal((c, 16))) for _ in range(layers)]


def test_wgrad_is_the_gradient_of_the_convolution():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 6, 3))
    dp = rng.standard_normal((2, 5, 6, 4))
    dw = T.conv3x3_wgrad(x, dp)
    for _ in range(3):
        V = rng.standard_normal((4, 3, 3, 3))
        assert abs(np.vdot(dw, V) - np.vdot(C.conv3x3(x, V), dp)) < 1e-10
    # one element by brute force: the corner tap reads x at (y-1, x-1)
    s = sum(dp[b, y, xx, 2] * x[b, y - 1, xx - 1, 1]
            for b in range(2) for y in range(1, 5) for xx in range(1, 6))
    assert abs(dw[2, 0, 0, 1] - s) < 1e-12


def test_channel_sum_is_the_bias_gradient():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 5, 3))
    dp = rng.standard_normal((1, 4, 5, 2))
    c = rng.standard_normal(2)
    lin = np.vdot(C.conv3x3(x, np.zeros((2, 3, 3, 3)), c), dp)
    assert abs(np.vdot(T.channel_sum(dp), c) - lin) < 1e-12


def test_dsm_loss_is_the_weighted_score_matching_integrand():
    rng = np.random.default_rng(3)
    x0, z, eps = (rng.standard_normal((2, 4, 5)) for _ in range(3))
    abar = 0.37
    x = T.noisy(x0, z, abar)
    # the conditional score of the Gaussian transition, and s = -eps / sigma
    cond = -(x - np.sqrt(abar) * x0) / (1.0 - abar)
    s = -eps / np.sqrt(1.0 - abar)
    weighted = (1.0 - abar) * np.sum((s - cond) ** 2)
    loss, g = T.dsm_loss(eps, z)
    assert abs(loss * eps.size - weighted) < 1e-10 * weighted
    # the gradient of a quadratic: central differences are exact up to rounding
    e = 1e-4
    d = np.zeros_like(eps)
    d[1, 2, 3] = e
    fd = (T.dsm_loss(eps + d, z)[0] - T.dsm_loss(eps - d, z)[0]) / (2 * e)
    assert abs(fd - g[1, 2, 3]) < 1e-10
    l0, g0 = T.dsm_loss(z, z)
    assert l0 == 0.0 and not np.any(g0)


def test_minibatch_gradient_matches_central_differences():
    w = _weights()
    rng = np.random.default_rng(4)
    x0 = rng.standard_normal((2, 5, 6))
    z = rng.standard_normal((2, 5, 6))
    abar, t = 0.6, 123
    loss, grads = T.dsm_gradients(w, x0, z, abar, t, round_bf16=False)

    def f(ws):
        return T.dsm_gradients(ws, x0, z, abar, t, round_bf16=False)[0]

    e = 1e-6
    probes = [(0, 0, (1, 2, 0, 0)), (1, 0, (3, 0, 2, 1)), (2, 0, (0, 1, 1, 3)),
              (0, 1, (2,)), (2, 1, (0,)), (1, 2, (1, 5)), (2, 2, (0, 9))]
    for l, k, idx in probes:
        plus = [list(p) for p in w]
        minus = [list(p) for p in w]
        plus[l][k] = np.array(w[l][k], np.float64)
        minus[l][k] = np.array(w[l][k], np.float64)
        plus[l][k][idx] += e
        minus[l][k][idx] -= e
        fd = (f(plus) - f(minus)) / (2 * e)
        got = grads[l][k][idx]
        assert abs(fd - got) <= 1e-7 * max(1.0, abs(fd)), (l, k, idx, fd, got)


def test_adam_closed_forms():
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(7)
    g = rng.standard_normal(7)
    lr, eps = 1e-2, 1e-8
    # with a constant gradient the bias-corrected moments are g and g^2 at
    # every step, so every step moves by lr g / (|g| + eps)
    p, m, v = p0, np.zeros(7), np.zeros(7)
    for t in range(1, 6):
        q, m, v = T.adam(p, g, m, v, t, lr, 0.9, 0.999, eps)
        np.testing.assert_allclose(p - q, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        p = q
    # the first moment is the discounted sum of the gradients
    gs = rng.standard_normal((4, 7))
    m = v = np.zeros(7)
    p = p0
    for t in range(1, 5):
        p, m, v = T.adam(p, gs[t - 1], m, v, t, lr)
    np.testing.assert_allclose(m, sum(0.1 * 0.9 ** (4 - k) * gs[k - 1] for k in range(1, 5)),
                               rtol=1e-13)
    np.testing.assert_allclose(v, sum(0.001 * 0.999 ** (4 - k) * gs[k - 1] ** 2
                                      for k in range(1, 5)), rtol=1e-12)


def test_time_bias_at_step_zero():
    rng = np.random.default_rng(6)
    b = rng.standard_normal(5)
    E = rng.standard_normal((5, 16))
    # phi(0) = [0 (sines), 1 (cosines)]
    np.testing.assert_allclose(T.time_bias(b, E, N.time_features(0)), b + E[:, 8:].sum(axis=1),
                               rtol=1e-14)


def test_regression_at_its_own_output_is_stationary():
    w = _weights(seed=7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 5, 6))
    y = N.ConvScore(w, round_bf16=False).eps(0.5 * x, 0)
    loss, grads = T.regression_gradients(w, x, y, 0, 0.5, round_bf16=False)
    assert loss == 0.0
    assert all(not np.any(g) for layer in grads for g in layer)
    # and a shifted target gives the loss of the shift
    loss2, _ = T.regression_gradients(w, x, y + 0.25, 0, 0.5, round_bf16=False)
    assert abs(loss2 - 0.0625) < 1e-12
