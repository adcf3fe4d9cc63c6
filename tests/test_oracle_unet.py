"""Pins of the U-Net oracle (``oracle/unet.py``), CPU only: pooling and
upsampling against brute force and their adjoint pairs (dot-product
identities), and the unrounded network's vector-Jacobian product and
parameter gradients against central differences."""
import numpy as np

from oracle import unet as U

WIDTHS = (2, 3, 4, 4)


def _weights(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for name, ci, co in U.layers(WIDTHS):
        out.append((rng.standard_normal((co, 3, 3, ci)) / np.sqrt(9 * ci),
                    0.1 * rng.standard_normal(co), 0.1 * rng.standard_normal((co, 16))))
    return out


def test_pool_and_upsample_by_brute_force():
    x = np.arange(2 * 5 * 3 * 1, dtype=np.float64).reshape(2, 5, 3, 1)
    y = U.pool2(x, 0)
    assert y.shape == (2, 3, 2, 1)
    assert y[0, 0, 0, 0] == (0 + 1 + 3 + 4) / 4          # full block
    assert y[0, 2, 1, 0] == x[0, 4, 2, 0]                 # corner: one cell
    assert y[1, 2, 0, 0] == (x[1, 4, 0, 0] + x[1, 4, 1, 0]) / 2
    assert U.pool2(x, 1)[0, 0, 0, 0] == 8
    u = U.up2(y, 5, 3, 0)
    assert u.shape == (2, 5, 3, 1) and u[0, 3, 2, 0] == y[0, 1, 1, 0]
    assert U.up2(y, 5, 3, 1)[0, 4, 2, 0] == y[0, 2, 1, 0]          # a one-cell block
    assert U.up2(y, 5, 3, 1)[0, 4, 0, 0] == y[0, 2, 0, 0] / 2


def test_resampling_adjoint_pairs():
    rng = np.random.default_rng(1)
    for h, w in ((6, 8), (5, 7), (1, 3)):
        x = rng.standard_normal((2, h, w, 3))
        g = rng.standard_normal((2, (h + 1) // 2, (w + 1) // 2, 3))
        # mean pooling and upsampling with the count division
        assert abs(np.vdot(U.pool2(x, 0), g) - np.vdot(x, U.up2(g, h, w, 1))) < 1e-12
        # nearest upsampling and sum pooling
        assert abs(np.vdot(U.up2(g, h, w, 0), x) - np.vdot(g, U.pool2(x, 1))) < 1e-12


def test_vjp_and_parameter_gradients_match_central_differences():
    w = _weights()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 9, 7))
    g = rng.standard_normal((1, 9, 7))
    t = 77
    net = U.UNet(w, WIDTHS, round_bf16=False)
    net.eps(x, t)
    u = net.backward(g)
    grads = net.param_grads(t)

    def f(ws, xx):
        return np.vdot(U.UNet(ws, WIDTHS, round_bf16=False).eps(xx, t), g)

    e = 1e-6
    for (i, j) in ((0, 0), (4, 3), (8, 6), (5, 1)):
        d = np.zeros_like(x)
        d[0, i, j] = e
        fd = (f(w, x + d) - f(w, x - d)) / (2 * e)
        assert abs(fd - u[0, i, j]) <= 1e-7 * max(1.0, abs(fd)), (i, j)
    names = [n for n, _, _ in U.layers(WIDTHS)]
    for name, k, idx in (("enc0a", 0, (1, 0, 2, 0)), ("enc3b", 0, (2, 1, 1, 3)),
                         ("dec2u", 0, (0, 2, 0, 1)), ("dec0c", 1, (1,)), ("out", 0, (0, 1, 1, 1)),
                         ("enc2a", 2, (3, 4)), ("dec1u", 1, (2,))):
        l = names.index(name)
        plus = [list(p) for p in w]
        minus = [list(p) for p in w]
        plus[l][k] = np.array(w[l][k], np.float64)
        minus[l][k] = np.array(w[l][k], np.float64)
        plus[l][k][idx] += e
        minus[l][k][idx] -= e
        fd = (f(plus, x) - f(minus, x)) / (2 * e)
        assert abs(fd - grads[l][k][idx]) <= 1e-7 * max(1.0, abs(fd)), (name, k, idx)
