"""The low-rank Gaussian prior on the GPU (fwi_lowrank_score_at) against the
FP64 oracle (oracle/diffusion.LowRankPrior): its score and the score's
vector-Jacobian product at device step indices, the isotropic case, the
out-of-range step, repeatability; and one graph-replayed reverse step of
Algorithm 2 driven by it (sampler.GraphChain) stage by stage against the
oracle's reverse step with the W2 potential."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_GRAD, models, problems, rel_l2  # noqa: E402
from oracle import diffusion as D  # noqa: E402
from oracle import oracle as O  # noqa: E402

DEV = "cuda:0"
N = 24
BETAS = D.linear_betas(N, 2e-3, 0.2)
SCHED = D.Schedule(BETAS)


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    return A, S


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def H(t):
    return t.double().cpu().numpy()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _prior(n=1024, k=6, seed=2, s2=0.01):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    U = f32(Q.T)
    return D.LowRankPrior(f32(rng.standard_normal(n) * 0.3), U, f32(rng.uniform(0.5, 4.0, k)),
                          s2), rng


@pytest.mark.parametrize("i", [1, 7, N])
def test_lowrank_score_and_vjp_match_oracle(mods, i):
    A, _ = mods
    pr, rng = _prior()
    B, n, k = 3, pr.mu.size, pr.U.shape[0]
    table = A.ddpm_table(list(BETAS), A.SIGMA_POSTERIOR, A.DiffusionSpace(), torch.device(DEV))
    step = torch.full((1,), i, dtype=torch.int32, device=DEV)
    x = f32(rng.standard_normal((B, n)))
    work = torch.empty(B * k, dtype=torch.float32, device=DEV)
    out = torch.empty((B, n), dtype=torch.float32, device=DEV)
    out2 = torch.empty_like(out)
    A.fwi_lowrank_score_at(B, n, T(pr.U), T(pr.lam), pr.s2, T(x), T(pr.mu), table, step, N,
                           work, out)
    A.fwi_lowrank_score_at(B, n, T(pr.U), T(pr.lam), pr.s2, T(x), T(pr.mu), table, step, N,
                           work, out2)
    torch.cuda.synchronize()
    ref = pr.score(x, SCHED.abar[i])
    assert rel_l2(H(out), ref) <= 1e-5, rel_l2(H(out), ref)
    assert torch.equal(out, out2)
    # the vector-Jacobian product applied to x (mu absent): -C^-1 x
    A.fwi_lowrank_score_at(B, n, T(pr.U), T(pr.lam), pr.s2, T(x), None, table, step, N, work,
                           out)
    torch.cuda.synchronize()
    assert rel_l2(H(out), pr.score_vjp(x, SCHED.abar[i])) <= 1e-5


def test_lowrank_isotropic_case_and_out_of_range_steps(mods):
    A, _ = mods
    pr, rng = _prior(k=3)
    B, n = 2, pr.mu.size
    table = A.ddpm_table(list(BETAS), A.SIGMA_POSTERIOR, A.DiffusionSpace(), torch.device(DEV))
    x = T(rng.standard_normal((B, n)))
    out = torch.zeros((B, n), dtype=torch.float32, device=DEV)
    step = torch.full((1,), 5, dtype=torch.int32, device=DEV)
    A.fwi_lowrank_score_at(B, n, None, None, 0.2, x, T(pr.mu), table, step, N, None, out)
    torch.cuda.synchronize()
    ref = D.gaussian_score(H(x), SCHED.abar[5], pr.mu, np.full(n, 0.2))
    assert rel_l2(H(out), ref) <= 1e-6
    for bad in (0, N + 1):     # outside 1..N nothing is written
        mark = torch.full((B, n), 7.0, dtype=torch.float32, device=DEV)
        step.fill_(bad)
        A.fwi_lowrank_score_at(B, n, T(pr.U), T(pr.lam), pr.s2, x, T(pr.mu), table, step, N,
                               torch.empty(B * 3, dtype=torch.float32, device=DEV), mark)
        torch.cuda.synchronize()
        assert bool((mark == 7.0).all())
    with pytest.raises(A.FwiError):
        A.fwi_lowrank_score_at(B, n, T(pr.U), T(pr.lam), 0.0, x, T(pr.mu), table, step, N,
                               torch.empty(B * 3, dtype=torch.float32, device=DEV), out)


def test_graph_chain_step_with_the_lowrank_prior_matches_oracle(mods):
    # one replayed reverse step (i = N) of Algorithm 2, W2 guidance
    A, S = mods
    B, nz, nx = 2, 32, 32
    gp, op = problems(nz, nx, 12, 300, 2, batch=B, f_peak=25.0)
    vt = models("curved_faulted", list(range(B)), nz, nx)
    d_obs = f32(O.forward(op, vt))
    fam = models("curved_faulted", list(range(40, 104)), nz, nx)
    prior = S.LowRankPrior.from_models(fam, k=12, device=torch.device(DEV))
    opr = D.LowRankPrior(H(prior.mu), H(prior.U), H(prior.lam), prior.s2)
    rng = np.random.default_rng(3)
    zs = f32(rng.standard_normal((N + 1, B, nz, nx)))
    v0 = f32(rng.standard_normal((B, nz, nx)))
    guide = A.GuideParams(rho0=2.0, c=1e9, gamma=0.5)
    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        chain = S.GraphChain(plan, BETAS, ctx, prior, guide, T(zs))
        v1 = chain.run(T(v0), N, N).clone()
        torch.cuda.synchronize()
        plan.check()
        w2p = O.W2Params()
        pot = D.w2_potential(op, O.w2_prepare(d_obs, op.dt, w2p), w2p)
        _, inter = D.reverse_step(SCHED, N, v0, zs[N], pot, None, None,
                                  O.GuideParams(rho0=2.0, c=1e9, gamma=0.5), prior=opr)
    assert rel_l2(H(chain.v0hat), inter["v0hat"]) <= 1e-5
    assert rel_l2(H(chain.v_prime), inter["v_prime"]) <= 1e-5
    assert rel_l2(H(chain.g), inter["g"]) <= TOL_GRAD
    assert rel_l2(H(chain.h), inter["h"]) <= TOL_GRAD
    assert np.isfinite(H(v1)).all()
    # the prior's samples are smooth: neighbouring cells of v0hat correlate
    v0h = inter["v0hat"]
    dx = np.diff(v0h, axis=2)
    assert np.std(dx) < 0.5 * np.std(v0h - v0h.mean())
