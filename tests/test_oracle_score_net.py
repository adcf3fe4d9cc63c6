"""Pins of the convolutional score model's oracle (``oracle/score_net.py``),
CPU only: the vector-Jacobian product against central differences of the
unrounded network, the transposed convolution against the dot-product
identity, SiLU's derivative against differences, and the bf16 rounding
against numpy's own float32 -> bfloat16 bit pattern rule on known values."""
import numpy as np

from oracle import conv as C
from oracle import score_net as N


def _weights(seed=0, c=8, layers=3):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((c, 3, 3, c)) / np.sqrt(9 * c), 0.1 * rng.standard_normal(c),
             0.1 * rng.standard_normal((c, 16))) for _ in range(layers)]


def test_vjp_matches_central_differences():
    net = N.ConvScore(_weights(), round_bf16=False)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 6, 7))
    g = rng.standard_normal((1, 6, 7))
    step = 321
    net.eps(x, step)
    u = net.eps_vjp(g)
    e = 1e-6
    fd = np.zeros_like(x)
    for i in range(6):
        for j in range(7):
            d = np.zeros_like(x)
            d[0, i, j] = e
            fd[0, i, j] = (np.vdot(net.eps(x + d, step), g) -
                           np.vdot(net.eps(x - d, step), g)) / (2 * e)
    assert np.linalg.norm(fd - u) <= 1e-7 * np.linalg.norm(fd)


def test_time_features_closed_form():
    f = N.time_features(0)
    np.testing.assert_array_equal(f, [0.0] * 8 + [1.0] * 8)
    f = N.time_features(7)
    assert f[0] == np.sin(7.0) and f[8] == np.cos(7.0)              # w_0 = 1
    np.testing.assert_allclose(f[:8] ** 2 + f[8:] ** 2, 1.0, rtol=0, atol=1e-15)
    assert abs(f[7] - np.sin(7 * 10000.0 ** (-7 / 8))) < 1e-15


def test_transposed_convolution_is_the_adjoint():
    rng = np.random.default_rng(2)
    w = rng.standard_normal((5, 3, 3, 4))
    x = rng.standard_normal((2, 6, 5, 4))
    y = rng.standard_normal((2, 6, 5, 5))
    wt = np.flip(w, axis=(1, 2)).transpose(3, 1, 2, 0)
    assert abs(np.vdot(C.conv3x3(x, w), y) - np.vdot(x, C.conv3x3(y, wt))) < 1e-10


def test_silu_derivative():
    p = np.linspace(-8, 8, 33)
    e = 1e-6
    fd = (N.silu(p + e) - N.silu(p - e)) / (2 * e)
    np.testing.assert_allclose(N.silu_grad(p), fd, rtol=0, atol=1e-8)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie (rounds to even, 1),
    # 3 + 2^-8 lies below half an ulp (2^-7) of 3,
    # 1 + 3 2^-9 rounds up to 1 + 2^-7, values already representable stay
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, -2.5, 3.0 + 2.0 ** -8, 0.0])
    np.testing.assert_array_equal(N.bf16(vals), [1.0, 1.0, 1 + 2.0 ** -7, -2.5, 3.0, 0.0])
    r = N.bf16(np.random.default_rng(3).standard_normal(1000))
    m, _ = np.frexp(r)
    assert np.all(np.abs(m * 2 ** 8 - np.round(m * 2 ** 8)) == 0)   # 8-bit significands
