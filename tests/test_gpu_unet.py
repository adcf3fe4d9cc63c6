"""GPU parity of the U-Net score network (``score_net.UNetScore``): the
resampling kernels against the FP64 oracle (``oracle/unet.py``), the
network's eps, vector-Jacobian product and DSM parameter gradients against
the oracle with the same bf16 storage points, a reverse step of Algorithm 2
driven by it, and DSM training that lowers the held-out loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import models, problems, rel_l2  # noqa: E402
from oracle import diffusion as D  # noqa: E402
from oracle import oracle as O  # noqa: E402
from oracle import score_net as N  # noqa: E402
from oracle import unet as U  # noqa: E402

DEV = "cuda:0"
BF16_ULP = 2.0 ** -8


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    from paper_2603_16393_gb300 import score_net as SN
    return A, S, SN


def F(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def BF(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32).to(torch.bfloat16).to(DEV)


def H(t):
    return t.double().cpu().numpy()


def _ulps(got, ref):
    """|got - ref| in units of bf16's spacing at ref (at least 2^-133)."""
    return np.abs(got - ref) / np.maximum(np.abs(ref) * BF16_ULP, 2.0 ** -133)


@pytest.mark.parametrize("h,w", [(33, 47), (8, 16), (1, 3)])
def test_resampling_kernels(mods, h, w):
    A, _, _ = mods
    rng = np.random.default_rng(h * w)
    c = 24
    x = N.bf16(rng.standard_normal((2, h, w, c)))
    hc, wc = (h + 1) // 2, (w + 1) // 2
    g = N.bf16(rng.standard_normal((2, hc, wc, c)))
    y = torch.empty((2, hc, wc, c), dtype=torch.bfloat16, device=DEV)
    u = torch.empty((2, h, w, c), dtype=torch.bfloat16, device=DEV)
    for mode in (0, 1):
        A.fwi_pool2_bf16(BF(x), y, mode)
        assert np.all(_ulps(H(y), N.bf16(U.pool2(x, mode))) <= 1.0)
        A.fwi_up2_bf16(BF(g), u, mode)
        ref = N.bf16(U.up2(g, h, w, mode))
        if mode == 0:
            np.testing.assert_array_equal(H(u), ref)
        else:
            assert np.all(_ulps(H(u), ref) <= 1.0)
    z = torch.empty((2, h, w, c), dtype=torch.bfloat16, device=DEV)
    A.fwi_add_bf16(BF(x), u, z)
    torch.cuda.synchronize()
    assert np.all(_ulps(H(z), N.bf16(x + H(u))) <= 1.0)


def test_unet_eps_vjp_and_dsm_gradients_match_oracle(mods):
    A, _, SN = mods
    B, nz, nx = 2, 33, 47
    betas = D.linear_betas(1000)
    widths = SN.UNET_WIDTHS
    w = SN.unet_seeded_weights(widths, seed=3)
    net = SN.UNetScore((B, nz, nx), betas, weights=w)
    ref = U.UNet(w, widths, round_bf16=True)
    exact = U.UNet(w, widths, round_bf16=False)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    i = 321
    e = net.eps(F(x), i)
    u = net.eps_vjp(F(g), 0.5)
    torch.cuda.synchronize()
    e_o = ref.eps(x, i)
    u_o = ref.backward(g, 0.5)
    # one bf16 ulp where the FP32-accumulated and the FP64 value round
    # differently, at any of the network's storage points
    err_e, err_u = rel_l2(H(e), e_o), rel_l2(H(u), u_o)
    assert err_e <= 8 * BF16_ULP, err_e
    assert err_u <= 8 * BF16_ULP, err_u
    assert rel_l2(H(e), exact.eps(x, i)) < 0.25
    # DSM gradients of a minibatch through the trainer
    tr = SN.DSMTrainer(net)
    z = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    t = 450
    loss = tr.gradients(F(x), F(z), t)
    torch.cuda.synchronize()
    l_ref, g_ref = U.dsm_gradients(w, widths, x, z, D.Schedule(betas).abar[t], t)
    assert abs(float(loss.item()) - l_ref) <= 5 * BF16_ULP * l_ref
    names = [n for n, _, _, _ in SN.unet_layers(widths)]
    for name, got, refl in zip(names, net.logical(tr.grads), g_ref):
        for k, what in enumerate(("W", "b", "E")):
            err = rel_l2(H(got[k]), refl[k])
            assert err <= 16 * BF16_ULP, (name, what, err)
    # a 32-channel level runs in a 64-channel block: the parameters of its
    # zero channels get exactly zero gradients, so training keeps them zero
    nz_pad = 0
    for (W, b, E), (_, _, ci, co) in zip(tr.grads, SN.unet_layers(widths)):
        nz_pad += int(torch.count_nonzero(W[co:])) + int(torch.count_nonzero(W[:, :, :, ci:]))
        nz_pad += int(torch.count_nonzero(b[co:])) + int(torch.count_nonzero(E[co:]))
    assert nz_pad == 0


def test_algorithm2_with_the_unet_score(mods):
    A, S, SN = mods
    B, nz, nx = 2, 32, 32
    gp, op = problems(nz, nx, 12, 300, 2, batch=B, f_peak=25.0)
    d_obs = O.forward(op, models("layered", [0, 1], nz, nx))
    betas = D.linear_betas(1000)
    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(F(d_obs))
        net = SN.UNetScore(plan.model_shape, betas)
        smp = S.Sampler(plan, betas, ctx=ctx, score_fn=net, guide=A.GuideParams(rho0=1.0))
        rng = np.random.default_rng(6)
        v = F(rng.standard_normal((B, nz, nx)) * 0.3)
        i = 250
        v_next, info = smp.step(v, i, F(rng.standard_normal((B, nz, nx))))
        torch.cuda.synchronize()
        plan.check()
        ab = smp.steps[i].abar
        uu = net.eps_vjp(smp.g, -1.0 / np.sqrt(1 - ab))
        h_ref = (H(smp.g) + (1 - ab) * H(uu)) / np.sqrt(ab)
        assert rel_l2(H(smp.h), h_ref) <= 1e-6
        assert torch.isfinite(v_next).all() and torch.isfinite(info["J"]).all()


def test_unet_training_lowers_the_held_out_loss(mods):
    A, _, SN = mods
    B, nz, nx = 8, 32, 32
    betas = D.linear_betas(1000)
    space = A.DiffusionSpace()
    v = models("layered", list(range(B)), nz, nx)
    x0 = F((v - space.shift) / space.unit)
    net = SN.UNetScore((B, nz, nx), betas, seed=2)
    tr = SN.DSMTrainer(net, lr=1e-3)
    assert tr.stage is not None           # every level's weight gradient on the tensor cores
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


@pytest.mark.parametrize("net_kind", ["unet", "conv"])
def test_full_batch_sampled_images_match_oracle(mods, net_kind):
    """152 models of 70 x 70 (the benchmark's batch and launch shapes): every
    layer acts on each image alone, so sampled images of eps and of the
    vector-Jacobian product are checked against the oracle run on them."""
    from oracle import score_net as NO
    A, _, SN = mods
    B, nz, nx = 152, 70, 70
    betas = D.linear_betas(1000)
    if net_kind == "unet":
        w = SN.unet_seeded_weights(SN.UNET_WIDTHS, seed=5)
        net = SN.UNetScore((B, nz, nx), betas, weights=w)
    else:
        w = SN.seeded_weights(128, 3, seed=5)
        net = SN.ConvScore((B, nz, nx), betas, weights=w)
    rng = np.random.default_rng(15)
    x = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    i = 640
    e = H(net.eps(F(x), i))
    u = H(net.eps_vjp(F(g), 1.0))
    torch.cuda.synchronize()
    for b in (0, 77, 151):
        if net_kind == "unet":
            ref = U.UNet(w, SN.UNET_WIDTHS, round_bf16=True)
            e_o = ref.eps(x[b:b + 1], i)
            u_o = ref.backward(g[b:b + 1], 1.0)
        else:
            ref = NO.ConvScore(w, round_bf16=True)
            e_o = ref.eps(x[b:b + 1], i)
            u_o = ref.eps_vjp(g[b:b + 1], 1.0)
        assert rel_l2(e[b:b + 1], e_o) <= 8 * BF16_ULP, (b, rel_l2(e[b:b + 1], e_o))
        assert rel_l2(u[b:b + 1], u_o) <= 8 * BF16_ULP, (b, rel_l2(u[b:b + 1], u_o))
