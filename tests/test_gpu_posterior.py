"""Algorithm 2 as a graph-replayed chain (sampler.GraphChain): the replayed
reverse steps are bitwise the eager Sampler's, the batched chain is bitwise
the plain path that runs one posterior sample per plan with eager launches
(so the two reconstruct equally well by construction), and the FD gate of the
surrogate phase checks, accepts and falls back on the device as it does on
the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import models, problems  # noqa: E402
from paper_2603_16393_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    from paper_2603_16393_gb300 import surrogate as SG
    return A, S, SG


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def _setup(A, S, B, nz=32, nx=32, nt=300, ns=2, N=24):
    gp, _ = problems(nz, nx, 10, nt, ns, batch=B, f_peak=25.0)
    plan = A.Plan(gp)
    d_obs = plan.forward(T(models("curved_faulted", list(range(B)), nz, nx)), store=False)[0].clone()
    ctx = plan.w2_prepare(d_obs)
    prior = S.GaussianPrior.from_models(I.model_batch("layered", range(50, 82), nz, nx),
                                        device=torch.device(DEV))
    betas = S.linear_betas(N, 2e-3, 0.2)
    gen = torch.Generator(device=DEV).manual_seed(7)
    zs = torch.randn((N + 1, B, nz, nx), device=DEV, generator=gen)
    v_start = torch.randn((B, nz, nx), device=DEV, generator=gen)
    return gp, plan, d_obs, ctx, prior, betas, zs, v_start


def test_replayed_chain_is_bitwise_the_eager_sampler(mods):
    A, S, _ = mods
    gp, plan, _, ctx, prior, betas, zs, v0 = _setup(A, S, 3)
    guide = A.GuideParams(rho0=1.0, gamma=0.5)
    chain = S.GraphChain(plan, betas, ctx, prior, guide, zs)
    v_graph = chain.run(v0).clone()
    smp = S.Sampler(plan, betas, ctx=ctx, prior=prior, guide=guide)
    v = v0
    for i in range(len(betas), 0, -1):
        v, _ = smp.step(v, i, zs[i])
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(v_graph, v)
    assert chain.counts == {"fd": len(betas), "sur": 0, "check": 0}
    assert int(chain.step.item()) == 0


def test_batched_chain_is_bitwise_the_plain_unbatched_path(mods):
    A, S, _ = mods
    B = 3
    gp, plan, d_obs, ctx, prior, betas, zs, v0 = _setup(A, S, B)
    guide = A.GuideParams(rho0=1.0, gamma=0.5)
    v_batched = S.GraphChain(plan, betas, ctx, prior, guide, zs).run(v0).clone()
    import dataclasses
    p1 = A.Plan(dataclasses.replace(gp, batch=1))
    for b in range(B):
        ctx1 = p1.w2_prepare(d_obs[b:b + 1].contiguous())
        smp = S.Sampler(p1, betas, ctx=ctx1, prior=prior, guide=guide)
        v = v0[b:b + 1].contiguous()
        for i in range(len(betas), 0, -1):
            v, _ = smp.step(v, i, zs[i, b:b + 1].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(v[0], v_batched[b]), b


class _Offset:
    """A stand-in surrogate: the FD gradient scaled by (1 + rel)."""

    def __init__(self, plan, ctx, rel):
        self.plan, self.ctx, self.rel = plan, ctx, rel

    def gradient(self, v_phys, stream=None, step=-1):
        J, g, _ = self.plan.gradient(v_phys, self.ctx, stream=stream)
        return J, g * (1.0 + self.rel)


@pytest.mark.parametrize("rel,accepted", [(0.02, True), (0.2, False)])
def test_device_gate_checks_and_falls_back(mods, rel, accepted):
    A, S, _ = mods
    gp, plan, _, ctx, prior, betas, zs, v0 = _setup(A, S, 2)
    guide = A.GuideParams(rho0=1.0, gamma=0.5)
    chain = S.GraphChain(plan, betas, ctx, prior, guide, zs, surrogate=_Offset(plan, ctx, rel),
                         surrogate_fraction=0.5, threshold=0.05, check_every=4)
    chain.run(v0)
    torch.cuda.synchronize()
    n_sur_phase = len(betas) - chain.i_switch
    if accepted:
        assert chain.counts["check"] == -(-n_sur_phase // 4)
        assert chain.counts["sur"] == n_sur_phase - chain.counts["check"]
        assert chain.counts["fd"] == chain.i_switch
        assert all(ok for _, _, ok in chain.records)
    else:
        assert chain.counts["check"] == 1 and chain.counts["sur"] == 0
        assert chain.counts["fd"] == len(betas) - 1
        assert chain.records[0][2] is False
    assert all(abs(e - rel) < 1e-5 for _, e, _ in chain.records)
