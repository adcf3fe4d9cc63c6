"""GPU parity of the reverse-diffusion loop (Algorithms 1-2, Sec. 4.2, 5.2):
the elementwise kernels, one and several reverse steps with the W2 and the
least-squares potentials, and the whole guidance-free chain, against the
FP64 oracle (``oracle/diffusion.py``) on the same seeded inputs and draws.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_GRAD, TOL_J, models, problems, rel_l2  # noqa: E402
from oracle import diffusion as D  # noqa: E402
from oracle import oracle as O  # noqa: E402

DEV = "cuda:0"
# float32 elementwise arithmetic against FP64: a few roundings of values of
# order one (the normalised space) or of order 1e3 (m/s)
TOL_ELEM = 2e-6


def update_error_bound(g, h, gp):
    """First-order bound on ||d(rho kappa h)|| / ||rho kappa h|| when g and h
    carry relative l2 errors up to TOL_GRAD (their own bar), from the
    oracle's g, h only: kappa_j = ((|g|_inf + eps) / (|g_j| + eps))^gamma
    multiplies dh_j by at most kappa_max, and its own relative change is
    gamma (|dg_j| / (|g_j| + eps) + d|g|_inf / (|g|_inf + eps))."""
    g, h = np.asarray(g, np.float64), np.asarray(h, np.float64)
    gmax = np.abs(g).max(axis=(1, 2), keepdims=True)
    kap = ((gmax + gp.eps) / (np.abs(g) + gp.eps)) ** gp.gamma
    nkh = np.linalg.norm(kap * h)
    m = (kap * np.abs(h) / (np.abs(g) + gp.eps)).max()
    return TOL_GRAD * (kap.max() * np.linalg.norm(h) + gp.gamma * m * np.linalg.norm(g)
                       + gp.gamma * nkh * np.linalg.norm(g) / (gmax.min() + gp.eps)) / nkh


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    return A, S


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def H(t):
    return t.double().cpu().numpy()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def close(a, b, tol=TOL_ELEM):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    err = np.abs(a - b)
    bound = tol * (np.abs(b) + np.abs(b).max())
    assert np.all(err <= bound), float((err / (np.abs(b) + np.abs(b).max())).max())


BETAS = D.linear_betas(1000)
SCHED = D.Schedule(BETAS)


@pytest.mark.parametrize("i", [1, 2, 150, 1000])
@pytest.mark.parametrize("given_score", [False, True])
def test_proposal_kernel_matches_oracle(mods, i, given_score):
    A, _ = mods
    rng = np.random.default_rng(i)
    B, nz, nx = 3, 37, 53                           # ragged: 5883 cells, not a multiple of 4
    v_i = f32(1.3 * rng.standard_normal((B, nz, nx)))
    z = f32(rng.standard_normal((B, nz, nx)))
    mu = f32(rng.uniform(-0.8, 0.8, (nz, nx)))
    tau2 = f32(rng.uniform(0.01, 0.4, (nz, nx)))
    s = f32(rng.standard_normal((B, nz, nx))) if given_score else None
    st = A.fwi_ddpm_coefficients(BETAS, i)
    sp = A.DiffusionSpace()
    out = [torch.empty((B, nz, nx), device=DEV) for _ in range(3)]
    A.fwi_ddpm_proposal(B, nz * nx, st, sp, T(v_i), T(s) if given_score else None, T(mu),
                        T(tau2), T(z), *out)
    torch.cuda.synchronize()
    ab = SCHED.abar[i]
    s_o = s if given_score else D.gaussian_score(v_i, ab, mu, tau2)
    x0 = D.clean_estimate(v_i, s_o, ab)
    close(H(out[0]), x0)
    close(H(out[1]), D.proposal(v_i, x0, z, SCHED, i))
    v_phys, mask = D.to_physical(x0)
    close(H(out[2]), v_phys)
    if given_score or i < 500:
        # both sides of the clamp are exercised (at high noise the prior's
        # clean estimate stays near mu, inside the clamp)
        assert 0 < mask.sum() < mask.size


@pytest.mark.parametrize("i", [2, 420, 1000])
@pytest.mark.parametrize("mode", ["prior", "vjp", "none"])
def test_guidance_kernel_matches_oracle(mods, mode, i):
    A, _ = mods
    rng = np.random.default_rng(7)
    B, nz, nx = 2, 29, 31
    x0 = f32(1.2 * rng.standard_normal((B, nz, nx)))
    g_phys = f32(1e-6 * rng.standard_normal((B, nz, nx)))
    tau2 = f32(rng.uniform(0.01, 0.4, (nz, nx)))
    u = f32(rng.standard_normal((B, nz, nx)))
    st = A.fwi_ddpm_coefficients(BETAS, i)
    g, h = torch.empty((B, nz, nx), device=DEV), torch.empty((B, nz, nx), device=DEV)
    A.fwi_ddpm_guidance(B, nz * nx, st, A.DiffusionSpace(), T(x0), T(g_phys),
                        T(u) if mode == "vjp" else None, T(tau2) if mode == "prior" else None,
                        g, h)
    torch.cuda.synchronize()
    ab = SCHED.abar[i]
    _, mask = D.to_physical(x0)
    g_o, _ = D.guidance_gradients(g_phys, mask, ab)
    uu = {"prior": D.gaussian_score_vjp(g_o, ab, tau2), "vjp": u, "none": None}[mode]
    g_o, h_o = D.guidance_gradients(g_phys, mask, ab, uu)
    close(H(g), g_o)
    close(H(h), h_o)
    assert np.all(H(g)[~np.broadcast_to(mask, g_o.shape)] == 0.0)


def _fwi_case(A, B=2, nz=32, nx=32, nt=300, ns=2):
    gp, op = problems(nz, nx, 12, nt, ns, batch=B, f_peak=25.0)
    vt = models("layered", list(range(B)), nz, nx)
    d_obs = O.forward(op, vt)
    fam = models("layered", list(range(20, 36)), nz, nx)
    mu = f32((fam.mean(axis=0) - D.SHIFT) / D.UNIT)
    tau2 = f32(np.maximum(((fam - D.SHIFT) / D.UNIT).var(axis=0), 0.02))
    return gp, op, d_obs, mu, tau2


def _state(i, B, nz, nx, mu, seed):
    rng = np.random.default_rng(seed)
    ab = SCHED.abar[i]
    return f32(np.sqrt(ab) * mu + np.sqrt(1 - ab) * rng.standard_normal((B, nz, nx)))


# rho0 large enough that the update stands well above the float32 rounding of v
GUIDE = O.GuideParams(rho0=2.0, c=0.1, tau=0.0, gamma=0.5, eps=1e-4)


def test_algorithm2_reverse_steps_match_oracle(mods):
    # three consecutive reverse steps with the W2 potential, on the same draws
    A, S = mods
    B, nz, nx = 2, 32, 32
    gp, op, d_obs, mu, tau2 = _fwi_case(A, B, nz, nx)
    w2p = O.W2Params()
    ctx_o = O.w2_prepare(d_obs, op.dt, w2p)
    pot = D.w2_potential(op, ctx_o, w2p)
    i0 = 300
    v = _state(i0, B, nz, nx, mu, 5)
    rng = np.random.default_rng(6)
    zs = {i: f32(rng.standard_normal((B, nz, nx))) for i in range(i0, i0 - 3, -1)}
    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        prior = S.GaussianPrior(T(mu), T(tau2))
        gparams = A.GuideParams(**{k: getattr(GUIDE, k) for k in
                                   ("rho0", "c", "tau", "gamma", "eps", "kappa_min", "kappa_max")})
        smp = S.Sampler(plan, BETAS, potential="w2", ctx=ctx, prior=prior, guide=gparams)
        v_gpu = T(v)
        v_or = v.copy()
        for k, i in enumerate(range(i0, i0 - 3, -1)):
            v_next, info = smp.step(v_gpu, i, T(zs[i]))
            torch.cuda.synchronize()
            plan.check()
            v_or_next, inter = D.reverse_step(SCHED, i, v_or, zs[i], pot, mu, tau2, GUIDE)
            if k == 0:
                # stage by stage on the first step (same input state)
                close(H(smp.v0hat), inter["v0hat"])
                close(H(smp.v_prime), inter["v_prime"])
                close(H(smp.v_phys), inter["v_phys"])
                assert rel_l2(H(info["J"]), inter["J"]) <= TOL_J
                assert rel_l2(H(smp.g), inter["g"]) <= TOL_GRAD
                assert rel_l2(H(smp.h), inter["h"]) <= TOL_GRAD
                assert rel_l2(H(info["rho"]), inter["rho"]) <= 1e-5
            # the guidance update P_i h: its error bound (x2) plus the float32
            # rounding of v_next = v' - P_i h (half an ulp of v_next)
            upd_o = v_or_next - inter["v_prime"]
            upd = H(v_next) - H(smp.v_prime)
            assert np.abs(upd_o).max() > 0
            bound = 2 * update_error_bound(inter["g"], inter["h"], GUIDE) * np.linalg.norm(upd_o) \
                + 2.0 ** -24 * np.linalg.norm(v_or_next)
            assert np.linalg.norm(upd - upd_o) <= bound, (k, np.linalg.norm(upd - upd_o), bound)
            # the state after k + 1 steps: each step adds at most its update's bound
            err_state = np.linalg.norm(H(v_next) - v_or_next)
            acc_bound = bound if k == 0 else acc_bound + bound + 2.0 ** -24 * np.linalg.norm(v_or)
            assert err_state <= 1.5 * acc_bound, (k, err_state, acc_bound)
            v_gpu, v_or = v_next, v_or_next


def test_algorithm1_dps_step_matches_oracle(mods):
    A, S = mods
    B, nz, nx = 2, 32, 32
    gp, op, d_obs, mu, tau2 = _fwi_case(A, B, nz, nx)
    sigma, zeta, i = 0.05, 3e-4, 120
    v = _state(i, B, nz, nx, mu, 8)
    z = f32(np.random.default_rng(9).standard_normal((B, nz, nx)))
    with A.Plan(gp) as plan:
        smp = S.Sampler(plan, BETAS, potential="l2", d_obs=T(d_obs), sigma_l2=sigma,
                        prior=S.GaussianPrior(T(mu), T(tau2)), dps_zeta=zeta)
        v_next, info = smp.step(T(v), i, T(z))
        torch.cuda.synchronize()
    v_o, inter = D.reverse_step(SCHED, i, v, z, D.l2_potential(op, d_obs, sigma), mu, tau2,
                                O.GuideParams(), dps_zeta=zeta)
    assert rel_l2(H(info["J"]), inter["J"]) <= TOL_J
    assert rel_l2(H(smp.h), inter["h"]) <= TOL_GRAD
    close(H(smp.v_prime), inter["v_prime"])
    upd_o = v_o - inter["v_prime"]                     # zeta h
    assert np.abs(upd_o).max() > 0
    # P_i = zeta I passes h's error through unchanged; plus the float32
    # rounding of v_next = v' - zeta h
    upd = H(v_next) - H(smp.v_prime)
    assert np.linalg.norm(upd - upd_o) <= TOL_GRAD * np.linalg.norm(upd_o) + \
        2.0 ** -24 * np.linalg.norm(v_o)
    np.testing.assert_array_equal(H(info["rho"]), np.float32(zeta))


def test_score_model_callback_matches_the_built_in_prior(mods):
    # a caller's score model (here the Gaussian prior written with torch ops
    # and torch.autograd for its vjp) gives the built-in prior's step
    A, S = mods
    B, nz, nx = 2, 32, 32
    gp, op, d_obs, mu, tau2 = _fwi_case(A, B, nz, nx)
    i = 250
    v = T(_state(i, B, nz, nx, mu, 3))
    z = T(np.random.default_rng(4).standard_normal((B, nz, nx)))
    mu_t, tau2_t = T(mu), T(tau2)
    ab = SCHED.abar[i]

    def score_fn(x, step):
        assert step == i
        xg = x.detach().requires_grad_(True)
        s = -(xg - np.sqrt(ab) * mu_t) / (ab * tau2_t + (1 - ab))

        def vjp(g):
            return torch.autograd.grad(s, xg, g, retain_graph=True)[0]

        return s.detach(), vjp

    with A.Plan(gp) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        gparams = A.GuideParams(rho0=0.05)
        a = S.Sampler(plan, BETAS, ctx=ctx, prior=S.GaussianPrior(mu_t, tau2_t), guide=gparams)
        va, _ = a.step(v, i, z)
        ha = a.h.clone()
        b = S.Sampler(plan, BETAS, ctx=ctx, score_fn=score_fn, guide=gparams)
        vb, _ = b.step(v, i, z)
        torch.cuda.synchronize()
    assert rel_l2(H(b.h), H(ha)) <= 1e-5
    assert np.abs(H(vb) - H(va)).max() <= 1e-5 * np.abs(H(va)).max()


def test_guidance_free_chain_matches_oracle_and_samples_the_prior(mods):
    # the whole reverse chain N..1 with no potential: elementwise against the
    # oracle on the same draws (a small batch), and the prior's first two
    # moments on a large batch
    A, S = mods
    nz, nx = 70, 70
    fam = models("layered", list(range(40)), nz, nx)
    x = (fam - D.SHIFT) / D.UNIT
    mu, tau2 = f32(x.mean(axis=0)), f32(np.maximum(x.var(axis=0), 0.01))
    gp, _ = problems(nz, nx, 40, 100, 1, batch=2)
    rng = np.random.default_rng(12)
    v0 = f32(rng.standard_normal((2, nz, nx)))
    zs = {i: f32(rng.standard_normal((2, nz, nx))) for i in range(1, SCHED.N + 1)}
    with A.Plan(gp) as plan:
        smp = S.Sampler(plan, BETAS, potential=None, prior=S.GaussianPrior(T(mu), T(tau2)))
        out = smp.sample(T(v0), lambda i: T(zs[i]))
        torch.cuda.synchronize()
    xo = v0.copy()
    for i in range(SCHED.N, 0, -1):
        ab = SCHED.abar[i]
        x0 = D.clean_estimate(xo, D.gaussian_score(xo, ab, mu, tau2), ab)
        xo = D.proposal(xo, x0, zs[i], SCHED, i)
    assert np.abs(H(out) - xo).max() <= 1e-4, np.abs(H(out) - xo).max()

    Bl = 128
    gpl, _ = problems(nz, nx, 40, 100, 1, batch=Bl)
    gen = torch.Generator(device=DEV).manual_seed(1)
    with A.Plan(gpl) as plan:
        smp = S.Sampler(plan, BETAS, potential=None, prior=S.GaussianPrior(T(mu), T(tau2)))
        start = torch.randn((Bl, nz, nx), device=DEV, generator=gen)
        out = smp.sample(start, lambda i: torch.randn((Bl, nz, nx), device=DEV, generator=gen))
        torch.cuda.synchronize()
    r = (H(out) - mu) / np.sqrt(tau2)
    assert abs(r.mean()) < 4 / np.sqrt(r.size), r.mean()
    assert abs(r.var() - 1) < 0.03, r.var()
