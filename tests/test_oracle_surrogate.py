"""Pins of the forward-surrogate oracle (oracle/surrogate.py) against what the
mathematics fixes: the trace map and its inverse, the adjoint pairs of the
pooling and upsampling along the image, the one-column convolution (and the
independence of models placed side by side, which the GPU's packing relies
on), the geometry channels, and the network's vector-Jacobian product and
parameter gradients against central differences of the unrounded network."""
import numpy as np
import pytest

from oracle import conv as C
from oracle import surrogate as S


def test_trace_map_round_trip_and_derivative():
    rng = np.random.default_rng(0)
    d = rng.standard_normal(200) * np.logspace(-6, 1, 200)
    amp = 3e-3
    np.testing.assert_allclose(S.slog_inv(S.slog(d, amp), amp), d, rtol=1e-12, atol=1e-18)
    y = rng.standard_normal(50) * 3.0
    h = 1e-6
    fd = (S.slog_inv(y + h, amp) - S.slog_inv(y - h, amp)) / (2 * h)
    np.testing.assert_allclose(fd, amp * np.exp(np.abs(y)), rtol=1e-7)
    assert S.slog(0.0, amp) == 0.0 and S.slog_inv(0.0, amp) == 0.0


@pytest.mark.parametrize("h", [1, 2, 5, 8, 35, 70])
def test_pool_and_upsampling_along_the_image(h):
    rng = np.random.default_rng(h)
    x = rng.standard_normal((2, h, 3, 4))
    p = S.pool_h(x, 0)
    for I in range(p.shape[1]):        # brute force: mean of the rows inside
        rows = [i for i in (2 * I, 2 * I + 1) if i < h]
        np.testing.assert_allclose(p[:, I], x[:, rows].mean(axis=1), rtol=1e-14)
    g = rng.standard_normal(p.shape)
    # <pool mean x, g> = <x, up_div g>; <up x, G> = <x, pool_sum G>
    assert np.isclose(np.sum(p * g), np.sum(x * S.up_h(g, h, 1)), rtol=1e-12)
    G = rng.standard_normal(x.shape)
    assert np.isclose(np.sum(S.up_h(g, h, 0) * G), np.sum(g * S.pool_h(G, 1)), rtol=1e-12)


def test_one_column_convolution_and_side_by_side_models():
    rng = np.random.default_rng(1)
    n, h, m, cin, cout = 2, 9, 4, 5, 3
    w3 = rng.standard_normal((cout, 3, cin))
    b = rng.standard_normal(cout)
    x = rng.standard_normal((n, h, m, cin))      # m models side by side
    y = C.conv3x3(x, S.expand_taps(w3), b)
    # brute force per model: y[i] = b + sum_k W3[k] x[i + k - 1] (zero outside)
    for j in range(m):
        for i in range(h):
            ref = b.copy()
            for k in range(3):
                if 0 <= i + k - 1 < h:
                    ref = ref + x[:, i + k - 1, j, :] @ w3[:, k, :].T
            np.testing.assert_allclose(y[:, i, j, :], ref, rtol=1e-12, atol=1e-12)
    # the models do not see each other: each alone gives the same result
    for j in range(m):
        yj = C.conv3x3(x[:, :, j:j + 1, :], S.expand_taps(w3), b)
        np.testing.assert_allclose(y[:, :, j:j + 1, :], yj, rtol=1e-13, atol=1e-13)


def test_geometry_channels():
    G = S.geometry_channels(4, 6, [0, 5], 16)
    assert G.shape == (6, 16)
    assert np.all(G[:, :4] == 0) and np.all(G[:, 9:] == 0)
    np.testing.assert_allclose(G[:, 4], (np.arange(6) - 0) / 6)
    np.testing.assert_allclose(G[:, 7], np.abs(np.arange(6) - 5) / 6)
    assert np.all(G[:, 8] == 1.0)
    with pytest.raises(ValueError):
        S.geometry_channels(10, 6, [0, 5], 12)


def _tiny(seed=0, round_bf16=False):
    nz, nx, nt, src, rec = 5, 7, 4, [1, 5], [0, 2, 3, 6]
    c0, width = 16, 8
    cout = len(src) * nt
    rng = np.random.default_rng(seed)
    w = S.seeded_weights(c0, width, cout, seed)
    w = [(W * 2.0, rng.standard_normal(b.shape) * 0.1) for W, b in w]   # exercise every term
    net = S.Surrogate(w, nz, nx, nt, src, rec, amp=0.5, c0=c0, in_scale=0.7, in_shift=-0.2,
                      round_bf16=round_bf16)
    return net, w, rng


def test_vjp_against_central_differences():
    net, _, rng = _tiny()
    v = rng.standard_normal((2, net.nz, net.nx))
    adj = rng.standard_normal((2, net.ns, net.nr, net.nt))
    net.forward(v)
    g = net.vjp(adj, scale=1.5)
    fd = np.zeros_like(v)
    h = 1e-6
    for idx in np.ndindex(*v.shape):
        vp, vm = v.copy(), v.copy()
        vp[idx] += h
        vm[idx] -= h
        fd[idx] = 1.5 * np.sum((net.forward(vp) - net.forward(vm)) * adj) / (2 * h)
    assert np.linalg.norm(g - fd) / np.linalg.norm(fd) < 1e-7


def test_parameter_gradients_against_central_differences():
    net, w, rng = _tiny(3)
    v = rng.standard_normal((2, net.nz, net.nx))
    d = rng.standard_normal((2, net.ns, net.nr, net.nt)) * 0.3
    loss, grads = S.training_gradients(net, v, d)

    def loss_at(ws):
        n2 = S.Surrogate(ws, net.nz, net.nx, net.nt, net.src_ix, net.rec_ix, net.amp, net.c0,
                         net.in_scale, net.in_shift, round_bf16=False)
        return S.regression_loss(n2.output(v), n2.target(d))[0]

    h = 1e-6
    for l in range(len(w)):
        for which in (0, 1):
            arr = w[l][which]
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(3)]:
                def bumped(delta):
                    ws = [(np.array(W, np.float64), np.array(b, np.float64)) for W, b in w]
                    ws[l][which][idx] += delta
                    return ws
                fd = (loss_at(bumped(h)) - loss_at(bumped(-h))) / (2 * h)
                assert np.isclose(grads[l][which][idx], fd, rtol=1e-6, atol=1e-10), \
                    (S.LAYERS[l], which, idx)


def test_target_inverts_the_trace_map_at_the_receivers():
    net, _, rng = _tiny(5)
    v = rng.standard_normal((1, net.nz, net.nx))
    d = net.forward(v)
    Yt = net.target(d)
    for x in net.rec_ix:
        np.testing.assert_allclose(Yt[:, x], net.Y[:, x], rtol=1e-10, atol=1e-12)
    others = [x for x in range(net.nx) if x not in net.rec_ix]
    assert np.all(Yt[:, others] == 0)
