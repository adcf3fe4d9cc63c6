"""Pins of the 3x3 convolution oracle (``oracle/conv.py``), CPU only: scipy's
2D cross-correlation summed over input channels, brute-force loops, kernels
with a closed-form result (identity, one-cell shifts with the zero border),
the SiLU through scipy's logistic function, and the sampled form."""
import numpy as np
import pytest
from scipy import signal, special

from oracle import conv as C


def _data(seed, n, h, w, cin, cout):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, h, w, cin)), rng.standard_normal((cout, 3, 3, cin)),
            rng.standard_normal(cout))


@pytest.mark.parametrize("shape", [(2, 7, 9, 3, 4), (1, 1, 1, 2, 2), (1, 5, 2, 4, 1)])
def test_matches_scipy_cross_correlation(shape):
    x, w, b = _data(1, *shape)
    n, h, wd, cin, cout = shape
    y = C.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for bb in range(n):
        for co in range(cout):
            acc = np.full((h, wd), b[co])
            for ci in range(cin):
                acc += signal.correlate2d(x[bb, :, :, ci], w[co, :, :, ci], mode="same",
                                          boundary="fill", fillvalue=0.0)
            ref[bb, :, :, co] = acc
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


def test_matches_brute_force_loops():
    x, w, b = _data(2, 1, 4, 5, 2, 3)
    y = C.conv3x3(x, w, b, act=1)
    for iy in range(4):
        for ix in range(5):
            for co in range(3):
                s = b[co]
                for ky in range(3):
                    for kx in range(3):
                        yy, xx = iy + ky - 1, ix + kx - 1
                        if 0 <= yy < 4 and 0 <= xx < 5:
                            for ci in range(2):
                                s += x[0, yy, xx, ci] * w[co, ky, kx, ci]
                assert abs(y[0, iy, ix, co] - s * special.expit(s)) < 1e-12


def test_identity_and_shift_kernels():
    x, _, _ = _data(3, 2, 6, 7, 4, 4)
    eye = np.zeros((4, 3, 3, 4))
    eye[:, 1, 1, :] = np.eye(4)
    np.testing.assert_array_equal(C.conv3x3(x, eye), x)
    up = np.zeros((4, 3, 3, 4))
    up[:, 0, 1, :] = np.eye(4)            # tap (ky-1, kx-1) = (-1, 0): y[iy] = x[iy - 1]
    y = C.conv3x3(x, up)
    np.testing.assert_array_equal(y[:, 1:], x[:, :-1])
    np.testing.assert_array_equal(y[:, 0], 0.0)
    right = np.zeros((4, 3, 3, 4))
    right[:, 1, 2, :] = np.eye(4)         # (0, +1): y[ix] = x[ix + 1]
    y = C.conv3x3(x, right)
    np.testing.assert_array_equal(y[:, :, :-1], x[:, :, 1:])
    np.testing.assert_array_equal(y[:, :, -1], 0.0)


def test_sampled_form_and_abs_sum():
    x, w, b = _data(4, 2, 5, 6, 3, 5)
    y = C.conv3x3(x, w, b, act=1)
    pix = [(0, 0, 0), (1, 4, 5), (1, 2, 3), (0, 4, 0)]
    ch = [4, 0, 2]
    got = C.conv3x3_at(x, w, b, 1, pix, ch)
    for k, (bb, iy, ix) in enumerate(pix):
        np.testing.assert_allclose(got[k], y[bb, iy, ix, ch], rtol=0, atol=1e-12)
    s = C.abs_sum(x, w)
    assert np.all(s >= np.abs(C.conv3x3(x, w)) - 1e-12)
