"""Pins of the oracle's reverse-diffusion loop (Sec. 3.3-3.5, 4.2, 5.2;
Algorithms 1-2), CPU only.

Each pin checks the oracle against something other than its own formulas:
numerical integration of the Gaussian densities the formulas come from
(marginal score, Tweedie's clean estimate, the Gaussian posterior of the
proposal), a Monte-Carlo run of the whole reverse chain, central differences
of the composite potential Phi(x0hat(v_i)), and the paper's statement that
P_i = zeta I turns Algorithm 2's step into the DPS step of Algorithm 1.
"""
import numpy as np
import pytest

from oracle import diffusion as D
from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I


def _grid(lo, hi, n=40001):
    x = np.linspace(lo, hi, n)
    return x, x[1] - x[0]


def _normal(x, m, var):
    return np.exp(-0.5 * (x - m) ** 2 / var) / np.sqrt(2 * np.pi * var)


SCHED = D.Schedule(D.linear_betas(1000))


@pytest.mark.parametrize("i", [1, 40, 300, 999])
def test_gaussian_score_is_the_log_derivative_of_the_marginal(i):
    # p_i(x) = int N(x; sqrt(abar) x0, 1 - abar) N(x0; mu, tau2) dx0 by
    # quadrature over x0; score = d/dx log p_i by central differences
    abar = SCHED.abar[i]
    mu, tau2 = 0.3, 0.2
    x0, dx0 = _grid(mu - 12 * np.sqrt(tau2), mu + 12 * np.sqrt(tau2))
    prior = _normal(x0, mu, tau2)

    def logp(x):
        return np.log(np.sum(_normal(x, np.sqrt(abar) * x0, 1 - abar) * prior) * dx0)

    for x in (-1.2, 0.1, 0.9):
        e = 1e-4
        fd = (logp(x + e) - logp(x - e)) / (2 * e)
        assert abs(D.gaussian_score(x, abar, mu, tau2) - fd) < 1e-6 * max(1.0, abs(fd))
        # the Jacobian of the score: second derivative of log p
        fd2 = (logp(x + e) - 2 * logp(x) + logp(x - e)) / e ** 2
        assert abs(D.gaussian_score_vjp(1.0, abar, tau2) - fd2) < 1e-4 * abs(fd2)


@pytest.mark.parametrize("i", [2, 60, 500, 1000])
def test_clean_estimate_is_the_posterior_mean(i):
    # Tweedie: Eq. v0hat with the exact score is E[x0 | x_i], computed here by
    # quadrature of x0 q(x_i | x0) p(x0)
    abar = SCHED.abar[i]
    mu, tau2 = -0.4, 0.35
    x0, dx0 = _grid(mu - 12 * np.sqrt(tau2), mu + 12 * np.sqrt(tau2))
    prior = _normal(x0, mu, tau2)
    for x in (-2.0, -0.3, 0.0, 1.5):
        w = _normal(x, np.sqrt(abar) * x0, 1 - abar) * prior
        post_mean = np.sum(x0 * w) / np.sum(w)
        est = D.clean_estimate(x, D.gaussian_score(x, abar, mu, tau2), abar)
        assert abs(est - post_mean) < 1e-8 * max(1.0, abs(post_mean)), (x, est, post_mean)


@pytest.mark.parametrize("i", [2, 10, 250, 1000])
def test_proposal_is_the_gaussian_posterior_of_the_previous_state(i):
    # q(x_{i-1} | x_i, x0) ∝ N(x_i; sqrt(alpha_i) x_{i-1}, beta_i) N(x_{i-1}; sqrt(abar_{i-1}) x0,
    # 1 - abar_{i-1}): mean and standard deviation by quadrature over x_{i-1}
    a, b, abp = SCHED.alpha[i], SCHED.beta[i], SCHED.abar[i - 1]
    for xi, x0 in ((0.7, -0.2), (-1.1, 0.5), (0.0, 0.9)):
        c = np.sqrt(abp) * x0
        lo, hi = min(c, xi / np.sqrt(a)) - 1.0, max(c, xi / np.sqrt(a)) + 1.0
        xp, dxp = _grid(lo, hi, 400001)
        # in logs: each factor alone can underflow where the product does not
        lw = -0.5 * (xi - np.sqrt(a) * xp) ** 2 / b - 0.5 * (xp - c) ** 2 / (1 - abp)
        w = np.exp(lw - lw.max())
        m = np.sum(xp * w) / np.sum(w)
        var = np.sum((xp - m) ** 2 * w) / np.sum(w)
        p0 = D.proposal(xi, x0, 0.0, SCHED, i)
        p1 = D.proposal(xi, x0, 1.0, SCHED, i)
        assert abs(p0 - m) < 1e-7, (p0, m)
        assert abs((p1 - p0) - np.sqrt(var)) < 1e-6 * np.sqrt(var), (p1 - p0, np.sqrt(var))


def test_last_step_returns_the_clean_estimate():
    # abar_0 = 1: the i = 1 proposal is x0hat itself (no noise)
    c_v, c_0, sg = SCHED.proposal_coefficients(1)
    assert c_v == 0.0 and sg == 0.0
    assert abs(c_0 - 1.0) < 1e-12     # beta_1 / (1 - (1 - beta_1)) in FP64
    beta_sched = D.Schedule(D.linear_betas(1000), sigma="beta")
    assert beta_sched.sigma[1] == np.sqrt(SCHED.beta[1])


def test_reverse_chain_samples_the_gaussian_prior():
    # Algorithm 2 with no guidance (rho0 = 0) and the exact score: the reverse
    # chain started from N(0, I) ends (up to the discretisation of 1000 steps)
    # with samples of the prior N(mu, tau2), per cell
    rng = np.random.default_rng(11)
    M = 60000
    mu = np.where(np.arange(M) % 2 == 0, 0.4, -0.6)
    tau2 = np.where(np.arange(M) % 2 == 0, 0.09, 0.25)
    x = rng.standard_normal(M)
    for i in range(SCHED.N, 0, -1):
        ab = SCHED.abar[i]
        x0 = D.clean_estimate(x, D.gaussian_score(x, ab, mu, tau2), ab)
        x = D.proposal(x, x0, rng.standard_normal(M), SCHED, i)
    for parity in (0, 1):
        s = x[parity::2]
        m, t = mu[parity], tau2[parity]
        assert abs(s.mean() - m) < 4 * np.sqrt(t / s.size), (s.mean(), m)
        assert abs(s.var() / t - 1) < 0.03, (s.var(), t)


def test_to_physical_clamps_and_masks():
    v, mask = D.to_physical(np.array([-1.2, -1.0, 0.0, 0.5, 1.0, 1.01]))
    np.testing.assert_array_equal(v, [1500, 1500, 3000, 3750, 4500, 4500])
    np.testing.assert_array_equal(mask, [False, True, True, True, True, False])


def _tiny(B=1):
    g = I.surface_geometry(12, 1)
    prob = O.Problem(nz=12, nx=12, nb=4, nt=90, dz=10.0, dx=10.0, dt=1e-3,
                     src_iz=g.src_iz, src_ix=g.src_ix, rec_iz=g.rec_iz, rec_ix=g.rec_ix,
                     f_peak=40.0, v_ref=2500.0)
    w2p = O.W2Params(n_xi=200)
    vt = 1800 + 400 * I.layered_model(1, 12, 12) / 4500.0 + I.smooth_perturbation(5, 12, 12, 150)
    ctx = O.w2_prepare(O.forward(prob, np.stack([vt] * B)), prob.dt, w2p)
    return prob, w2p, ctx


def test_guidance_gradient_matches_central_differences_of_the_composite():
    # Eq. chain_rule: h = d/dv_i Phi(x0hat(v_i)) with x0hat = (v_i + (1 - abar)
    # s(v_i)) / sqrt(abar), Phi = J of the clamped physical model; central
    # differences of that composite at every cell, some of them clamped
    prob, w2p, ctx = _tiny()
    i = 200
    abar = SCHED.abar[i]
    mu = (2100 + I.smooth_perturbation(8, 12, 12, 200) - D.SHIFT) / D.UNIT
    tau2 = np.full((12, 12), 0.04)
    rng = np.random.default_rng(4)
    v_i = np.sqrt(abar) * mu + 0.05 * rng.standard_normal((12, 12))
    v_i[0, 3] = -40.0       # far below: x0hat clamped at v_lo
    potential = D.w2_potential(prob, ctx, w2p, threads=1)

    def composite(vi):
        x0 = D.clean_estimate(vi, D.gaussian_score(vi, abar, mu, tau2), abar)
        vph, _ = D.to_physical(x0)
        return potential(vph[None])[0][0]

    _, inter = D.reverse_step(SCHED, i, v_i[None], np.zeros((1, 12, 12)), potential, mu, tau2,
                              O.GuideParams())
    h = inter["h"][0]
    assert not inter["mask"][0][0, 3] and inter["mask"][0].sum() == 143
    e = 1e-6
    fd = np.zeros_like(v_i)
    for iz in range(12):
        for ix in range(12):
            d = np.zeros_like(v_i)
            d[iz, ix] = e
            fd[iz, ix] = (composite(v_i + d) - composite(v_i - d)) / (2 * e)
    assert fd[0, 3] == 0.0 and h[0, 3] == 0.0
    rel = np.linalg.norm(fd - h) / np.linalg.norm(fd)
    assert rel < 1e-6, rel


def test_dps_step_is_algorithm_2_with_a_scalar_preconditioner():
    # Sec. 5.2: with P_i = zeta I the preconditioned step is the DPS step;
    # gamma = 0 gives kappa = 1 and an unreachable tau gives rho = rho0 = zeta
    prob, w2p, ctx = _tiny(B=2)
    i, zeta = 37, 0.02
    rng = np.random.default_rng(9)
    mu = (2300 + I.smooth_perturbation(2, 12, 12, 200) - D.SHIFT) / D.UNIT
    tau2 = np.full((12, 12), 0.1)
    v_i = rng.standard_normal((2, 12, 12)) * 0.2 + mu
    z = rng.standard_normal((2, 12, 12))
    pot = D.w2_potential(prob, ctx, w2p, threads=1)
    a, _ = D.reverse_step(SCHED, i, v_i, z, pot, mu, tau2,
                          O.GuideParams(rho0=zeta, gamma=0.0, tau=1e30))
    b, inter = D.reverse_step(SCHED, i, v_i, z, pot, mu, tau2, O.GuideParams(), dps_zeta=zeta)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15 * np.abs(b).max())
    assert np.abs(inter["h"]).max() > 0


def _lowrank(n=36, k=5, seed=3, s2=0.05):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return D.LowRankPrior(rng.standard_normal(n) * 0.3, Q.T, rng.uniform(0.2, 3.0, k), s2), rng


@pytest.mark.parametrize("abar", [1e-4, 0.03, 0.5, 0.999])
def test_lowrank_score_against_the_dense_covariance(abar):
    # brute force: the step-i marginal's covariance abar Sigma + (1 - abar) I
    # formed as a dense matrix, its score by a linear solve
    pr, rng = _lowrank()
    n = pr.mu.size
    Sig = pr.U.T @ np.diag(pr.lam) @ pr.U + pr.s2 * np.eye(n)
    C = abar * Sig + (1.0 - abar) * np.eye(n)
    x = rng.standard_normal((3, n))
    ref = -np.linalg.solve(C, (x - np.sqrt(abar) * pr.mu).T).T
    np.testing.assert_allclose(pr.score(x, abar), ref, rtol=1e-10, atol=1e-12)
    # Tweedie: the clean estimate is the Gaussian conditional mean
    # E[x0 | x] = mu + Cov(x0, x) Var(x)^-1 (x - E x), Cov(x0, x) = sqrt(abar) Sigma
    post = pr.mu + (np.sqrt(abar) * Sig @ np.linalg.solve(C, (x - np.sqrt(abar) * pr.mu).T)).T
    np.testing.assert_allclose(D.clean_estimate(x, pr.score(x, abar), abar), post,
                               rtol=1e-8, atol=1e-8)


def test_lowrank_score_vjp_and_the_diagonal_special_case():
    pr, rng = _lowrank(seed=5)
    n, abar = pr.mu.size, 0.2
    x, g = rng.standard_normal((1, n)), rng.standard_normal((1, n))
    # (ds/dx)^T g against central differences of <s(x), g>
    h = 1e-6
    fd = np.array([(np.sum(pr.score(x + h * e, abar) * g) - np.sum(pr.score(x - h * e, abar) * g))
                   / (2 * h) for e in np.eye(n)[:, None, :]])
    np.testing.assert_allclose(pr.score_vjp(g, abar)[0], fd, rtol=1e-6, atol=1e-9)
    # no correlated directions: the diagonal prior with tau2 = s2
    flat = D.LowRankPrior(pr.mu, np.zeros((0, n)), np.zeros(0), 0.3)
    np.testing.assert_allclose(flat.score(x, abar),
                               D.gaussian_score(x, abar, pr.mu, np.full(n, 0.3)), rtol=1e-14)
