"""GPU parity of denoising-score-matching training (Eq. L2_rewrite) of the
convolutional score model: the weight gradient, channel sum, DSM loss, Adam,
weight preparation and per-step bias kernels against the FP64 oracle
(``oracle/score_train.py``), the trainer's minibatch gradients against the
oracle's chain rule with the same bf16 storage points, a sampled check of
the weight gradient at the size the benchmark trains on, and a short
training run that lowers the held-out DSM loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import models, rel_l2  # noqa: E402
from oracle import diffusion as D  # noqa: E402
from oracle import score_net as N  # noqa: E402
from oracle import score_train as T  # noqa: E402

DEV = "cuda:0"
U32 = 2.0 ** -24          # float32 unit roundoff
BF16_ULP = 2.0 ** -8


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import score_net as SN
    return A, SN


def F(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def BF(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32).to(torch.bfloat16).to(DEV)


def H(t):
    return t.double().cpu().numpy()


def _bf16_pair(rng, shape):
    """Seeded values exactly representable in bf16 (the oracle sees what the GPU sees)."""
    return N.bf16(rng.standard_normal(shape)), N.bf16(rng.standard_normal(shape))


@pytest.mark.parametrize("n,h,w,c,use_work", [(2, 33, 47, 64, True), (2, 33, 47, 64, False),
                                              (1, 9, 13, 128, True), (1, 5, 7, 192, True)])
def test_weight_gradient_and_channel_sum(mods, n, h, w, c, use_work):
    A, _ = mods
    rng = np.random.default_rng(n * 1000 + c)
    x, dp = _bf16_pair(rng, (n, h, w, c))
    dW = torch.empty((c, 3, 3, c), dtype=torch.float32, device=DEV)
    work = torch.empty(A.WGRAD_MAX_SPLITS * 9 * c * c, dtype=torch.float32, device=DEV) \
        if use_work else None
    X, dP = BF(x), BF(dp)
    A.fwi_conv3x3_wgrad(X, dP, dW, work)
    db = torch.empty(c, dtype=torch.float32, device=DEV)
    A.fwi_channel_sum(dP, db, work)
    torch.cuda.synchronize()
    ref = T.conv3x3_wgrad(x, dp)
    # a float32 sum of exact bf16 x bf16 products: |err| <= m u sum|terms|,
    # m the additions along one output's chain (pixels and splits)
    npix = n * h * w
    scale = T.conv3x3_wgrad(np.abs(x), np.abs(dp))
    err = np.abs(H(dW) - ref)
    assert np.all(err <= (npix + 16) * U32 * scale + 1e-30), err.max()
    # the transposed-operand mistake would show: the tap read at (y-1, x-1)
    assert rel_l2(H(dW), ref) < 1e-5
    err_b = np.abs(H(db) - T.channel_sum(dp))
    # chain: a range's pixels per lane, the lanes, the ranges
    assert np.all(err_b <= (npix + 1024) * U32 * T.channel_sum(np.abs(dp)) + 1e-30)
    # a fixed summation order: a second launch is bit-identical
    dW2 = torch.empty_like(dW)
    A.fwi_conv3x3_wgrad(X, dP, dW2, work)
    assert torch.equal(dW, dW2)


# (1, 2, 70): 5 blocks of 64 padded pixels; room for 4 ranges, 3 used (2, 2, 1)
@pytest.mark.parametrize("n,h,w,c,splits", [(2, 33, 47, 128, 32), (2, 33, 47, 128, 0),
                                            (1, 9, 13, 256, 32), (3, 5, 70, 128, 32),
                                            (1, 2, 70, 128, 4), (2, 33, 47, 64, 32),
                                            (1, 9, 13, 192, 32)])
def test_weight_gradient_on_the_tensor_cores(mods, n, h, w, c, splits):
    A, _ = mods
    rng = np.random.default_rng(n * 7 + c + w)
    x, dp = _bf16_pair(rng, (n, h, w, c))
    X, dP = BF(x), BF(dp)
    dW = torch.empty((c, 3, 3, c), dtype=torch.float32, device=DEV)
    stage = torch.empty(A.fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, c, c), dtype=torch.uint8,
                        device=DEV)
    work = torch.empty(splits * 9 * c * c, dtype=torch.float32, device=DEV) if splits else None
    if splits == 4:
        assert A.fwi_conv3x3_wgrad_tc_splits(n, h, w, c, c, work.numel()) == 3
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    dW.fill_(float("nan"))
    A.fwi_conv3x3_wgrad_tc(X, dP, dW, stage, work, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = T.conv3x3_wgrad(x, dp)
    # exact bf16 products, FP32 accumulation in an order the hardware picks
    # along the padded pixels Q, then the splits
    wp = (w + 2 + 7) // 8 * 8
    Q = n * (h + 2) * wp
    scale = T.conv3x3_wgrad(np.abs(x), np.abs(dp))
    err = np.abs(H(dW) - ref)
    assert np.all(err <= 2 * (Q + 64) * U32 * scale + 1e-30), err.max()
    assert rel_l2(H(dW), ref) < 1e-5
    dW2 = torch.empty_like(dW)
    A.fwi_conv3x3_wgrad_tc(X, dP, dW2, stage, work, status)
    assert torch.equal(dW, dW2)


@pytest.mark.parametrize("cin,cout", [(64, 128), (128, 64), (256, 128), (64, 192)])
@pytest.mark.parametrize("impl", ["cuda_cores", "tensor_cores"])
def test_weight_gradient_with_unequal_channels(mods, impl, cin, cout):
    A, _ = mods
    n, h, w = 2, 17, 24
    rng = np.random.default_rng(cin + 7 * cout)
    x = N.bf16(rng.standard_normal((n, h, w, cin)))
    dp = N.bf16(rng.standard_normal((n, h, w, cout)))
    dW = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device=DEV)
    work = torch.empty(A.WGRAD_MAX_SPLITS * 9 * cin * cout, dtype=torch.float32, device=DEV)
    if impl == "cuda_cores":
        A.fwi_conv3x3_wgrad(BF(x), BF(dp), dW, work)
        chain = n * h * w + 16
    else:
        stage = torch.empty(A.fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, cin, cout),
                            dtype=torch.uint8, device=DEV)
        A.fwi_conv3x3_wgrad_tc(BF(x), BF(dp), dW, stage, work)
        chain = 2 * (n * (h + 2) * 32 + 64)
    torch.cuda.synchronize()
    ref = T.conv3x3_wgrad(x, dp)
    scale = T.conv3x3_wgrad(np.abs(x), np.abs(dp))
    assert np.all(np.abs(H(dW) - ref) <= chain * U32 * scale + 1e-30)
    assert rel_l2(H(dW), ref) < 1e-5


@pytest.mark.parametrize("impl", ["cuda_cores", "tensor_cores"])
def test_weight_gradient_sampled_at_the_benchmark_size(mods, impl):
    """152 models of 70 x 70 at 128 channels (the training benchmark's batch),
    16 pixel ranges: sampled outputs summed one by one in FP64."""
    A, _ = mods
    n, h, w, c = 152, 70, 70, 128
    rng = np.random.default_rng(11)
    x = rng.standard_normal((n, h, w, c), dtype=np.float32)
    dp = rng.standard_normal((n, h, w, c), dtype=np.float32)
    X = torch.from_numpy(x).to(torch.bfloat16).to(DEV)
    dP = torch.from_numpy(dp).to(torch.bfloat16).to(DEV)
    del x, dp
    xb, pb = X.float().cpu().numpy(), dP.float().cpu().numpy()      # the bf16 values, exact
    dW = torch.empty((c, 3, 3, c), dtype=torch.float32, device=DEV)
    work = torch.empty(A.WGRAD_MAX_SPLITS * 9 * c * c, dtype=torch.float32, device=DEV)
    if impl == "cuda_cores":
        assert A.fwi_conv3x3_wgrad_splits(n, h, w, c, c, work.numel()) > 1
        A.fwi_conv3x3_wgrad(X, dP, dW, work)
        chain = n * h * w + 16
    else:
        assert A.fwi_conv3x3_wgrad_tc_splits(n, h, w, c, c, work.numel()) > 1
        stage = torch.empty(A.fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, c, c), dtype=torch.uint8,
                            device=DEV)
        A.fwi_conv3x3_wgrad_tc(X, dP, dW, stage, work)
        chain = 2 * (n * (h + 2) * 72 + 64)
    torch.cuda.synchronize()
    got = H(dW)
    for co, ky, kx, ci in [(0, 0, 0, 0), (127, 2, 2, 127), (5, 1, 1, 77), (64, 0, 2, 3),
                           (99, 2, 0, 64), (31, 1, 0, 32)]:
        xs = np.zeros((n, h + 2, w + 2))
        xs[:, 1:h + 1, 1:w + 1] = xb[..., ci]
        a = pb[..., co].astype(np.float64).ravel()
        b = xs[:, ky:ky + h, kx:kx + w].ravel()
        ref = float(a @ b)
        bound = chain * U32 * float(np.abs(a) @ np.abs(b))
        assert abs(got[co, ky, kx, ci] - ref) <= bound, (co, ky, kx, ci)


def test_dsm_noisy_and_loss(mods):
    A, _ = mods
    rng = np.random.default_rng(3)
    shape = (2, 33, 47)
    x0, z, eps = (rng.standard_normal(shape).astype(np.float32).astype(np.float64)
                  for _ in range(3))
    abar = 0.4137
    xt = torch.empty(shape, dtype=torch.float32, device=DEV)
    A.fwi_dsm_noisy(F(x0), F(z), abar, xt)
    ref = T.noisy(x0, z, abar)
    mag = np.sqrt(abar) * np.abs(x0) + np.sqrt(1 - abar) * np.abs(z)
    assert np.all(np.abs(H(xt) - ref) <= 3 * U32 * mag)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    g = torch.empty(shape, dtype=torch.float32, device=DEV)
    l_ref, g_ref = T.dsm_loss(eps, z)
    for work in (None, torch.empty(1024, dtype=torch.float32, device=DEV)):
        A.fwi_dsm_loss(F(eps), F(z), loss, g, work)
        torch.cuda.synchronize()
        assert abs(float(loss.item()) - l_ref) <= 1e-5 * l_ref
    assert np.all(np.abs(H(g) - g_ref) <= 4 * U32 * (np.abs(eps) + np.abs(z)) * 2 / eps.size)
    A.fwi_dsm_loss(F(z), F(z), loss, g)
    assert float(loss.item()) == 0.0 and not torch.any(g)


def test_adam_weight_prep_and_time_bias(mods):
    A, _ = mods
    rng = np.random.default_rng(4)
    n = 10007
    p = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    P, M, V = F(p), torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    m = v = np.zeros(n)
    lr = 2e-3
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        A.fwi_adam_step(P, F(g), M, V, step, lr)
        p, m, v = T.adam(p, g, m, v, step, lr)
    torch.cuda.synchronize()
    assert np.all(np.abs(H(P) - p) <= 3 * (2 * U32 * np.abs(p) + 1e-5 * lr))
    assert np.all(np.abs(H(M) - m) <= 1e-6 * np.abs(m).max())
    assert np.all(np.abs(H(V) - v) <= 1e-6 * np.abs(v).max())
    # bf16 weights and their transpose: bit-exact
    for cout, cin in ((64, 64), (128, 64)):
        w = rng.standard_normal((cout, 3, 3, cin)).astype(np.float32)
        Wb = torch.empty((cout, 3, 3, cin), dtype=torch.bfloat16, device=DEV)
        WTb = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=DEV)
        A.fwi_conv3x3_weights_prep(F(w), Wb, WTb)
        torch.cuda.synchronize()
        wr = N.bf16(w)
        np.testing.assert_array_equal(H(Wb), wr)
        np.testing.assert_array_equal(H(WTb), np.flip(wr, axis=(1, 2)).transpose(3, 1, 2, 0))
    # per-step biases and their E gradient
    c, steps = 64, 1001
    b = rng.standard_normal(c).astype(np.float32).astype(np.float64)
    E = (0.1 * rng.standard_normal((c, 16))).astype(np.float32).astype(np.float64)
    phi = np.stack([N.time_features(i) for i in range(steps)]).astype(np.float32).astype(np.float64)
    out = torch.empty((steps, c), dtype=torch.float32, device=DEV)
    A.fwi_time_bias(F(b), F(E), F(phi), out)
    ref = T.time_bias(b, E, phi)
    scale = np.abs(b) + np.abs(phi) @ np.abs(E).T
    db = F(rng.standard_normal(c))
    dE = torch.empty((c, 16), dtype=torch.float32, device=DEV)
    A.fwi_time_bias_grad(db, F(phi[700]), dE)
    torch.cuda.synchronize()
    assert np.all(np.abs(H(out) - ref) <= 17 * U32 * scale)
    np.testing.assert_allclose(H(dE), np.outer(H(db), phi[700]), rtol=U32, atol=0)


@pytest.mark.parametrize("c", [64, 128])     # 128: the tensor-core weight gradient
def test_minibatch_gradients_match_oracle(mods, c):
    A, SN = mods
    B, nz, nx = 2, 33, 47
    betas = D.linear_betas(1000)
    w = SN.seeded_weights(c, 3, seed=7)
    net = SN.ConvScore((B, nz, nx), betas, weights=w)
    tr = SN.DSMTrainer(net)
    assert tr.stage is not None           # the weight gradient on the tensor cores
    rng = np.random.default_rng(8)
    x0 = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    z = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    t = 300
    loss = tr.gradients(F(x0), F(z), t)
    torch.cuda.synchronize()
    l_ref, g_ref = T.dsm_gradients(w, x0, z, D.Schedule(betas).abar[t], t, round_bf16=True)
    assert abs(float(loss.item()) - l_ref) <= 5 * BF16_ULP * l_ref
    exact = T.dsm_gradients(w, x0, z, D.Schedule(betas).abar[t], t, round_bf16=False)[1]
    for l, (got, ref, ex) in enumerate(zip(tr.grads, g_ref, exact)):
        for k, name in enumerate(("W", "b", "E")):
            e = rel_l2(H(got[k]), ref[k])
            # the bf16 storage points of the forward and backward passes
            assert e <= 8 * BF16_ULP, (l, name, e)
            assert rel_l2(H(got[k]), ex[k]) < 0.25, (l, name)


def test_training_lowers_the_held_out_loss(mods):
    A, SN = mods
    B, nz, nx, c = 8, 32, 32, 64
    betas = D.linear_betas(1000)
    space = A.DiffusionSpace()
    v = models("layered", list(range(B)), nz, nx)
    x0 = F((v - space.shift) / space.unit)
    net = SN.ConvScore((B, nz, nx), betas, channels=c, seed=1)
    tr = SN.DSMTrainer(net, lr=2e-3)
    rng = np.random.default_rng(9)
    held = [(int(t), F(rng.standard_normal((B, nz, nx)))) for t in (50, 250, 500, 900)]

    def held_out():
        return float(np.mean([tr.gradients(x0, zz, t).item() for t, zz in held]))

    before = held_out()
    for _ in range(150):
        t = int(rng.integers(1, 1001))
        tr.step(x0, F(rng.standard_normal((B, nz, nx))), t)
    torch.cuda.synchronize()
    after = held_out()
    assert np.isfinite(after) and torch.isfinite(net.theta).all()
    assert after < 0.7 * before, (before, after)


def test_regression_gradients_match_oracle(mods):
    A, SN = mods
    B, nz, nx, c = 2, 33, 47, 64
    betas = D.linear_betas(1000)
    w = SN.seeded_weights(c, 3, seed=12)
    net = SN.ConvScore((B, nz, nx), betas, weights=w)
    tr = SN.DSMTrainer(net)
    v = models("layered", [3, 4], nz, nx)
    rng = np.random.default_rng(13)
    y = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    s = 1.0 / 3000.0
    loss = tr.regression_gradients(F(v), F(y), 0, s)
    torch.cuda.synchronize()
    l_ref, g_ref = T.regression_gradients(w, v, y, 0, s)
    assert abs(float(loss.item()) - l_ref) <= 5 * BF16_ULP * l_ref
    for l, (got, ref) in enumerate(zip(tr.grads, g_ref)):
        for k in range(3):
            assert rel_l2(H(got[k]), ref[k]) <= 8 * BF16_ULP, (l, k)


def test_network_surrogate_trained_on_fd_pairs(mods):
    """A convolutional surrogate of dJ/dv trained on pairs the FD path
    generates, then standing in for the physics in Algorithm 2's first steps."""
    A, SN = mods
    from gpu_cases import problems
    from paper_2603_16393_gb300 import sampler as S
    from oracle import oracle as O
    B, nz, nx = 4, 32, 32
    gp, op = problems(nz, nx, 12, 300, 2, batch=B, f_peak=25.0)
    d_obs = O.forward(op, models("layered", list(range(B)), nz, nx))
    betas = D.linear_betas(1000)
    rng = np.random.default_rng(14)
    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(F(d_obs))
        # pairs: smoothed perturbations of a linear model and their W2 gradients
        pairs = []
        for _ in range(6):
            v = 2000.0 + 1500.0 * np.linspace(0, 1, nz)[None, :, None] * np.ones((B, 1, nx))
            v = v + 150.0 * rng.standard_normal((B, nz, nx))
            vt = F(v)
            _, g, _ = plan.gradient(vt, ctx)
            pairs.append((vt, g.clone()))
        torch.cuda.synchronize()
        out_scale = max(float(g.abs().max()) for _, g in pairs)
        ys = [(g / out_scale).contiguous() for _, g in pairs]
        net = SN.ConvScore((B, nz, nx), betas, channels=64, seed=3)
        tr = SN.DSMTrainer(net, lr=2e-3)
        s = 1.0 / 3000.0

        def loss_all():
            return float(np.mean([tr.regression_gradients(v, y, 0, s).item()
                                  for (v, _), y in zip(pairs, ys)]))

        before = loss_all()
        for k in range(200):
            j = k % len(pairs)
            tr.regression_step(pairs[j][0], ys[j], 0, s)
        torch.cuda.synchronize()
        after = loss_all()
        assert np.isfinite(after) and after < 0.5 * before, (before, after)
        sur = S.NetworkSurrogate(net, s, out_scale)
        smp = S.Sampler(plan, betas, ctx=ctx, prior=S.GaussianPrior(F(np.zeros((nz, nx))),
                                                                    F(np.full((nz, nx), 0.1))),
                        guide=A.GuideParams(rho0=1.0), surrogate=sur, surrogate_fraction=0.4)
        x = F(0.3 * rng.standard_normal((B, nz, nx)))
        z = F(rng.standard_normal((B, nz, nx)))
        v1, info1 = smp.step(x, 900, z)          # the surrogate's phase: no J
        v2, info2 = smp.step(x, 100, z)          # the physics' phase
        torch.cuda.synchronize()
        assert smp.uses_surrogate(900) and not smp.uses_surrogate(100)
        assert info1["J"] is None and torch.isfinite(info2["J"]).all()
        assert torch.isfinite(v1).all() and torch.isfinite(v2).all()
