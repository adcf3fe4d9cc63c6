"""GPU parity of the learned forward surrogate (``surrogate.ForwardSurrogate``):
its data-side kernels (packing, trace map and its transpose, regression
target and loss, pooling and upsampling along the image, three-tap weight
preparation and gradient extraction) against the FP64 oracle
(``oracle/surrogate.py``), and the network's seismograms, vector-Jacobian
product and training gradients against the oracle with the same bf16 storage
points -- on a small configuration with a ragged last image and on the
production sizes (70 x 70 models, 5 shots x 1000 samples)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import rel_l2  # noqa: E402
from oracle import score_net as N  # noqa: E402
from oracle import surrogate as OS  # noqa: E402

DEV = "cuda:0"
BF16_ULP = 2.0 ** -8


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import surrogate as S
    return A, S


def F(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def BF(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32).to(torch.bfloat16).to(DEV)


def H(t):
    return t.double().cpu().numpy()


def _ulps(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref) * BF16_ULP, 2.0 ** -133)


@pytest.mark.parametrize("h,w", [(70, 8), (35, 1), (9, 3), (1, 2)])
def test_resampling_along_the_image(mods, h, w):
    A, _ = mods
    rng = np.random.default_rng(h + 10 * w)
    c = 16
    x = N.bf16(rng.standard_normal((2, h, w, c)))
    hc = (h + 1) // 2
    g = N.bf16(rng.standard_normal((2, hc, w, c)))
    y = torch.empty((2, hc, w, c), dtype=torch.bfloat16, device=DEV)
    u = torch.empty((2, h, w, c), dtype=torch.bfloat16, device=DEV)
    for mode in (0, 1):
        A.fwi_pool_h_bf16(BF(x), y, mode)
        A.fwi_up_h_bf16(BF(g), u, mode)
        torch.cuda.synchronize()
        assert np.all(_ulps(H(y), N.bf16(OS.pool_h(x, mode))) <= 1.0)
        ref = N.bf16(OS.up_h(g, h, mode))
        if mode == 0:
            np.testing.assert_array_equal(H(u), ref)
        else:
            assert np.all(_ulps(H(u), ref) <= 1.0)


def test_three_tap_weights_and_their_gradient(mods):
    A, _ = mods
    rng = np.random.default_rng(0)
    co, ci = 128, 64
    w3 = rng.standard_normal((co, 3, ci)).astype(np.float32)
    Wb = torch.empty((co, 3, 3, ci), dtype=torch.bfloat16, device=DEV)
    WTb = torch.empty((ci, 3, 3, co), dtype=torch.bfloat16, device=DEV)
    A.fwi_sur_weights_prep(F(w3), Wb, WTb)
    dW = rng.standard_normal((co, 3, 3, ci)).astype(np.float32)
    dW3 = torch.empty((co, 3, ci), dtype=torch.float32, device=DEV)
    A.fwi_sur_wgrad_centre(F(dW), dW3)
    torch.cuda.synchronize()
    ref = N.bf16(OS.expand_taps(w3))
    np.testing.assert_array_equal(H(Wb), ref)
    np.testing.assert_array_equal(H(WTb), np.flip(ref, axis=(1, 2)).transpose(3, 1, 2, 0))
    np.testing.assert_array_equal(H(dW3), dW[:, :, 1, :])


def _small(S, nmod, m, seed=1):
    nz, nx, nt, src, rec = 12, 20, 60, [0, 9, 19], [0, 1, 3, 4, 7, 10, 12, 15, 18, 19]
    c0, width = 64, 64
    cout = -(-len(src) * nt // 256) * 256
    w = OS.seeded_weights(c0, width, cout, seed)
    rng = np.random.default_rng(seed)
    w = [(W * 2.0, (rng.standard_normal(b.shape) * 0.1).astype(np.float32)) for W, b in w]
    amp = 0.05
    net = S.ForwardSurrogate(nmod, nz, nx, nt, src, rec, amp, width=width, c0=c0, m=m,
                             weights=w)
    ref = OS.Surrogate(w, nz, nx, nt, src, rec, amp, c0, net.in_scale, net.in_shift,
                       round_bf16=True)
    v = (2500.0 + 800.0 * rng.standard_normal((nmod, nz, nx))).astype(np.float32)
    return net, ref, v.astype(np.float64), rng


def test_packing_and_input_gradient(mods):
    A, S = mods
    net, ref, v, rng = _small(S, 11, 4)
    net.forward(F(v))
    torch.cuda.synchronize()
    X = H(net.X0)                          # [nimg][nx][m][c0]
    Xo = N.bf16(ref.pack(v))               # [nmod][nx][1][c0]
    for b in range(11):
        np.testing.assert_array_equal(X[b // 4, :, b % 4, :], Xo[b, :, 0, :])
    assert np.all(X[2, :, 3, :] == 0)      # the column past the last model
    dX = rng.standard_normal(tuple(net.dX.shape)).astype(np.float32)
    dv = torch.empty(net.shape, dtype=torch.float32, device=DEV)
    A.fwi_sur_unpack_grad(F(dX), dv, 4, net.in_scale)
    torch.cuda.synchronize()
    for b in range(11):
        np.testing.assert_allclose(H(dv)[b], net.in_scale * dX[b // 4, :, b % 4, :12].T,
                                   rtol=1e-7)


@pytest.mark.parametrize("nmod,m", [(11, 4), (8, 8)])
def test_seismograms_and_vjp_match_oracle(mods, nmod, m):
    A, S = mods
    net, ref, v, rng = _small(S, nmod, m)
    d = net.forward(F(v))
    adj = rng.standard_normal((nmod, 3, 10, 60)).astype(np.float32).astype(np.float64)
    g = net.vjp(F(adj), 0.5)
    torch.cuda.synchronize()
    d_o = ref.forward(v)
    g_o = ref.vjp(adj, 0.5)
    # one bf16 ulp where the FP32-accumulated and the FP64 value round
    # differently at a storage point, carried through the trace map
    assert rel_l2(H(d), d_o) <= 8 * BF16_ULP, rel_l2(H(d), d_o)
    assert rel_l2(H(g), g_o) <= 8 * BF16_ULP, rel_l2(H(g), g_o)
    exact = OS.Surrogate([(W, b) for W, b in net.weights()], net.nz, net.nx, net.nt,
                         ref.src_ix, ref.rec_ix, net.amp, net.c0, net.in_scale, net.in_shift,
                         round_bf16=False)
    assert rel_l2(H(d), exact.forward(v)) < 0.1


def test_training_gradients_match_oracle(mods):
    A, S = mods
    net, ref, v, rng = _small(S, 8, 4, seed=5)
    tr = S.SurrogateTrainer(net)
    d = (0.3 * rng.standard_normal((8, 3, 10, 60))).astype(np.float32).astype(np.float64)
    loss = tr.gradients(F(v), F(d))
    torch.cuda.synchronize()
    l_ref, g_ref = OS.training_gradients(ref, v, d)
    assert abs(float(loss.item()) - l_ref) <= 4 * BF16_ULP * l_ref
    for name, got, refl in zip(OS.LAYERS, tr.grads, g_ref):
        for k, what in enumerate(("W3", "b")):
            err = rel_l2(H(got[k]), refl[k])
            assert err <= 16 * BF16_ULP, (name, what, err)


def test_production_sizes_sampled_models(mods):
    # the configuration the sampler and the bench use: 70 x 70 models, five
    # surface shots, receivers at every column, 1000 samples, 16 models in two
    # images of 8; models 0 and 13 against the oracle
    A, S = mods
    nz = nx = 70
    nt = 1000
    src, rec = [0, 17, 34, 52, 69], list(range(70))
    rng = np.random.default_rng(7)
    net = S.ForwardSurrogate(16, nz, nx, nt, src, rec, amp=0.02, seed=11)
    w = net.weights()
    v = (3000.0 + 900.0 * np.tanh(rng.standard_normal((16, nz, nx)))).astype(np.float32)
    adj = rng.standard_normal((16, 5, 70, nt)).astype(np.float32)
    d = net.forward(F(v))
    g = net.vjp(F(adj))
    torch.cuda.synchronize()
    pick = [0, 13]
    ref = OS.Surrogate(w, nz, nx, nt, src, rec, 0.02, 128, net.in_scale, net.in_shift,
                       round_bf16=True)
    d_o = ref.forward(v[pick].astype(np.float64))
    g_o = ref.vjp(adj[pick].astype(np.float64))
    assert rel_l2(H(d)[pick], d_o) <= 8 * BF16_ULP
    assert rel_l2(H(g)[pick], g_o) <= 8 * BF16_ULP


def test_relative_error_per_model(mods):
    # the FD check's measure: ||g_b - r_b|| / ||r_b|| per model, FP64 sums
    A, _ = mods
    rng = np.random.default_rng(3)
    r = rng.standard_normal((5, 70, 70)).astype(np.float32) * 1e-7
    g = r * (1.0 + rng.standard_normal(r.shape).astype(np.float32) * 0.3)
    r[3] = 0.0                       # zero reference: inf for a nonzero g ...
    g[4] = 0.0
    r[4] = 0.0                       # ... and 0 when both are zero
    e = A.fwi_rel_error(F(g), F(r))
    e2 = A.fwi_rel_error(F(g), F(r))
    torch.cuda.synchronize()
    gd, rd = g.astype(np.float64), r.astype(np.float64)
    ref = [np.linalg.norm(gd[b] - rd[b]) / np.linalg.norm(rd[b]) for b in range(3)]
    np.testing.assert_allclose(H(e)[:3], ref, rtol=1e-6)
    assert np.isinf(H(e)[3]) and H(e)[4] == 0.0
    assert torch.equal(e, e2)
