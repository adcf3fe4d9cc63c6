"""GPU parity of the convolutional score model (``score_net.ConvScore``) on
the tensor-core convolution: the elementwise kernels, the network's eps and
its vector-Jacobian product against the FP64 oracle with the same bf16
storage points, and Algorithm 2 driven by it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import problems, rel_l2  # noqa: E402
from oracle import diffusion as D  # noqa: E402
from oracle import oracle as O  # noqa: E402
from oracle import score_net as N  # noqa: E402

DEV = "cuda:0"
# one bf16 ulp (2^-8 relative) where the FP32-accumulated and the FP64 value
# round differently, at each of the network's storage points
BF16_ULP = 2.0 ** -8


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    from paper_2603_16393_gb300 import score_net as SN
    return A, S, SN


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def H(t):
    return t.double().cpu().numpy()


def test_elementwise_kernels(mods):
    A, _, _ = mods
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 7)).astype(np.float32)
    X = torch.full((2, 5, 7, 64), 7.0, dtype=torch.bfloat16, device=DEV)
    A.fwi_pack_channel0(T(x), X, 0.5)
    Xh = X.float().cpu().numpy()
    np.testing.assert_array_equal(Xh[..., 0], N.bf16(0.5 * x.astype(np.float64)))
    assert np.all(Xh[..., 1:] == 0)
    Y = T(rng.standard_normal((2, 5, 7, 64)))
    y = torch.empty((2, 5, 7), device=DEV)
    A.fwi_unpack_channel0(Y, y, -3.0)
    np.testing.assert_array_equal(H(y), (-3.0 * Y[..., 0].cpu().numpy()).astype(np.float64))
    # 4096: eight elements per thread (16-byte accesses); 4093: one per thread
    for m in (4096, 4093):
        p = torch.tensor(8 * rng.standard_normal(m), dtype=torch.float32).to(torch.bfloat16)
        da = torch.tensor(rng.standard_normal(m), dtype=torch.float32).to(torch.bfloat16)
        a, dp = torch.empty_like(p, device=DEV), torch.empty_like(p, device=DEV)
        A.fwi_silu_bf16(p.to(DEV), a)
        A.fwi_silu_grad_bf16(da.to(DEV), p.to(DEV), dp)
        ph, dah = p.double().numpy(), da.double().numpy()
        for got, ref in ((a, N.bf16(N.silu(ph))), (dp, N.bf16(dah * N.silu_grad(ph)))):
            err = np.abs(got.double().cpu().numpy() - ref)
            assert np.all(err <= BF16_ULP * np.abs(ref) + 1e-30)


@pytest.mark.parametrize("cout", [64, 128, 256])
def test_fused_silu_epilogue_is_the_two_pass_layer(mods, cout):
    # one launch writing p and SiLU(p) against the convolution (bf16 out)
    # followed by fwi_silu_bf16: the same bits, on a ragged image (tiles cut
    # at both edges), both kernel shapes (cout 256: pixels as M; 64, 128:
    # pixels as N, a 64-channel remainder on zero weight rows)
    A, _, _ = mods
    n, h, w, cin = 2, 19, 23, 128
    g = torch.Generator(device=DEV).manual_seed(cout)
    x = torch.randn((n, h, w, cin), device=DEV, generator=g).to(torch.bfloat16)
    wt = (0.05 * torch.randn((cout, 3, 3, cin), device=DEV, generator=g)).to(torch.bfloat16)
    bias = torch.randn(cout, device=DEV, generator=g)
    p1 = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device=DEV)
    a1 = torch.empty_like(p1)
    A.fwi_conv3x3_bf16(x, wt, bias, 0, p1)
    A.fwi_silu_bf16(p1, a1)
    p2 = torch.full_like(p1, 7.0)
    a2 = torch.full_like(p1, 7.0)
    A.fwi_conv3x3_bf16_silu(x, wt, bias, p2, a2)
    torch.cuda.synchronize()
    assert torch.equal(p1.view(torch.int16), p2.view(torch.int16))
    assert torch.equal(a1.view(torch.int16), a2.view(torch.int16))
    with pytest.raises(A.FwiError):           # act 2 needs the activation output
        A.fwi_conv3x3_bf16(x, wt, bias, 2, p1)


@pytest.mark.parametrize("cout", [64, 128, 256])
def test_fused_silu_grad_epilogue_is_the_two_pass_product(mods, cout):
    # the gradient convolution times SiLU' of the layer below in one launch
    # against the convolution (bf16 out) followed by fwi_silu_grad_bf16
    A, _, _ = mods
    n, h, w, cin = 2, 19, 23, 128
    g = torch.Generator(device=DEV).manual_seed(100 + cout)
    x = torch.randn((n, h, w, cin), device=DEV, generator=g).to(torch.bfloat16)
    wt = (0.05 * torch.randn((cout, 3, 3, cin), device=DEV, generator=g)).to(torch.bfloat16)
    p = (3 * torch.randn((n, h, w, cout), device=DEV, generator=g)).to(torch.bfloat16)
    d1 = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device=DEV)
    A.fwi_conv3x3_bf16(x, wt, None, 0, d1)
    A.fwi_silu_grad_bf16(d1, p, d1)
    d2 = torch.full_like(d1, 7.0)
    A.fwi_conv3x3_bf16_silu_grad(x, wt, p, d2)
    torch.cuda.synchronize()
    assert torch.equal(d1.view(torch.int16), d2.view(torch.int16))
    assert float(d2.float().abs().max()) > 0


@pytest.mark.parametrize("channels", [64, 128])
def test_network_and_vjp_match_oracle(mods, channels):
    A, _, SN = mods
    B, nz, nx = 2, 33, 47
    betas = D.linear_betas(1000)
    w = SN.seeded_weights(channels, 3, seed=4)
    net = SN.ConvScore((B, nz, nx), betas, weights=w)
    ref = N.ConvScore(w, round_bf16=True)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((B, nz, nx)).astype(np.float32).astype(np.float64)
    i = 300
    ab = D.Schedule(betas).abar[i]
    s, vjp = net(T(x), i)
    u = vjp(T(g))
    torch.cuda.synchronize()
    s_o = ref.score(x, ab, i)
    u_o = ref.score_vjp(g, ab)
    bound = 5 * BF16_ULP      # 2 (L - 1) + 1 storage points on either path
    assert rel_l2(H(s), s_o) <= bound, rel_l2(H(s), s_o)
    assert rel_l2(H(u), u_o) <= bound, rel_l2(H(u), u_o)
    # an unrounded FP64 network is farther than the bf16 twin: the bf16
    # storage points, not the tensor cores, set the difference
    exact = N.ConvScore(w, round_bf16=False)
    assert rel_l2(H(s), exact.score(x, ab, i)) < 0.1
    # the step enters through the biases: another step, another score
    s2, _ = net(T(x), 700)
    assert rel_l2(H(s2) * np.sqrt(1 - D.Schedule(betas).abar[700]),
                  H(s) * np.sqrt(1 - ab)) > 1e-3


def test_algorithm2_with_the_convolutional_score(mods):
    A, S, SN = mods
    from gpu_cases import models
    B, nz, nx = 2, 32, 32
    gp, op = problems(nz, nx, 12, 300, 2, batch=B, f_peak=25.0)
    d_obs = O.forward(op, models("layered", [0, 1], nz, nx))
    betas = D.linear_betas(1000)
    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        net = SN.ConvScore(plan.model_shape, betas)
        smp = S.Sampler(plan, betas, ctx=ctx, score_fn=net, guide=A.GuideParams(rho0=1.0))
        rng = np.random.default_rng(6)
        v = T(rng.standard_normal((B, nz, nx)) * 0.3)
        i = 250
        v_next, info = smp.step(v, i, T(rng.standard_normal((B, nz, nx))))
        torch.cuda.synchronize()
        plan.check()
        # the step used the network: h = (g + (1 - abar) (ds/dv)^T g) / sqrt(abar)
        ab = smp.steps[i].abar
        u = net.eps_vjp(smp.g, -1.0 / np.sqrt(1 - ab))
        h_ref = (H(smp.g) + (1 - ab) * H(u)) / np.sqrt(ab)
        assert rel_l2(H(smp.h), h_ref) <= 1e-6
        assert torch.isfinite(v_next).all() and torch.isfinite(info["J"]).all()
