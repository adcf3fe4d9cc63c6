"""FP64 oracle of the reverse-diffusion loop around the physics gradient
(Sec. 3.3-3.5, 4.2, 5.2): the clean estimate (Eq. v0hat), the DDPM proposal,
the chain rule of the guidance gradient (Eq. chain_rule) and one reverse step
of Algorithm 1 (DPS, least-squares potential) and of Algorithm 2 (OT-guided
preconditioned DPS).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
It shares no code with the CUDA binding.  Plain numpy in float64, one
formula per function, in the order Algorithm 2 takes the steps.

Readings (the paper leaves these open):
* Schedule: beta_1..beta_N are given; alpha_i = 1 - beta_i,
  abar_i = prod_{j <= i} alpha_j and abar_0 = 1 (Sec. 4.2).  ``linear_betas``
  is the linear schedule 1e-4 .. 0.02 of the DDPM formulation the method
  builds on; the paper fixes no values.
* sigma_i ("variance {sigma_i}" in Algorithms 1-2): the standard deviation of
  the Gaussian q(x_{i-1} | x_i, x_0), sqrt((1 - abar_{i-1}) beta_i / (1 - abar_i))
  (``sigma="posterior"``), or sqrt(beta_i) (``sigma="beta"``).
* Normalised space: the diffusion state is x = (v - shift) / unit with
  shift = 3000 and unit = 1500 m/s (velocities 1500..4500 map to [-1, 1]).
  The physics runs on v = clamp(shift + unit x0hat, v_lo, v_hi); the clamp
  keeps early, noisy estimates inside the propagator's stability bound, and
  its derivative is 1 for v_lo <= shift + unit x0hat <= v_hi, else 0.
* Score model: the trained U-Net needs the paper's data and weights, so the
  loop takes the score as an input.  The closed-form stand-in used here is a
  Gaussian prior x_0 ~ N(mu, diag tau2) in the normalised space: by
  Eq. vp_transition the marginal at step i is N(sqrt(abar_i) mu,
  abar_i tau2 + 1 - abar_i), whose score is
      s_i(x) = -(x - sqrt(abar_i) mu) / (abar_i tau2 + 1 - abar_i),
  with the diagonal Jacobian -1 / (abar_i tau2 + 1 - abar_i).  A second
  stand-in, LowRankPrior, correlates the cells along k principal directions
  (smooth samples, as a trained prior gives); its score follows from the
  same transition with a covariance of known eigenbasis.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

SHIFT, UNIT, V_LO, V_HI = 3000.0, 1500.0, 1500.0, 4500.0


def linear_betas(n: int, beta_1: float = 1e-4, beta_n: float = 0.02) -> np.ndarray:
    """beta_1..beta_N, linear (index 0 of the result is beta_1)."""
    return np.linspace(beta_1, beta_n, n, dtype=np.float64)


class Schedule:
    """alpha_i, abar_i (abar_0 = 1) and sigma_i for i = 1..N (Sec. 4.2)."""

    def __init__(self, betas, sigma: str = "posterior"):
        b = np.asarray(betas, dtype=np.float64)
        self.N = len(b)
        self.beta = np.concatenate([[0.0], b])            # beta[i], i = 1..N
        self.alpha = 1.0 - self.beta
        self.abar = np.ones(self.N + 1)
        for i in range(1, self.N + 1):
            self.abar[i] = self.abar[i - 1] * self.alpha[i]
        self.sigma = np.zeros(self.N + 1)
        for i in range(1, self.N + 1):
            if sigma == "posterior":
                var = (1.0 - self.abar[i - 1]) * self.beta[i] / (1.0 - self.abar[i])
            elif sigma == "beta":
                var = self.beta[i]
            else:
                raise ValueError(sigma)
            self.sigma[i] = np.sqrt(var)

    def proposal_coefficients(self, i: int):
        """(c_v, c_0, sigma_i): v' = c_v v_i + c_0 v0hat + sigma_i z (Algorithms 1-2)."""
        ab, abp = self.abar[i], self.abar[i - 1]
        c_v = np.sqrt(self.alpha[i]) * (1.0 - abp) / (1.0 - ab)
        c_0 = np.sqrt(abp) * self.beta[i] / (1.0 - ab)
        return c_v, c_0, self.sigma[i]


def gaussian_score(x, abar: float, mu, tau2):
    """Score of the step-i marginal of the Gaussian prior N(mu, diag tau2)."""
    x, mu, tau2 = (np.asarray(a, dtype=np.float64) for a in (x, mu, tau2))
    return -(x - np.sqrt(abar) * mu) / (abar * tau2 + 1.0 - abar)


def gaussian_score_vjp(g, abar: float, tau2):
    """(d s_i / d x)^T g for the Gaussian prior (a diagonal Jacobian)."""
    g, tau2 = np.asarray(g, dtype=np.float64), np.asarray(tau2, dtype=np.float64)
    return -g / (abar * tau2 + 1.0 - abar)


class LowRankPrior:
    """x_0 ~ N(mu, Sigma), Sigma = U diag(lam) U^T + s2 I, U [k][n] with
    orthonormal rows: a Gaussian prior with k correlated directions (the
    principal components of a set of models) over an isotropic floor.  By
    Eq. vp_transition the step-i marginal is N(sqrt(abar) mu, C),
    C = abar Sigma + (1 - abar) I, whose eigenvalues are
    c_j = abar (lam_j + s2) + 1 - abar along row j of U and
    c_perp = abar s2 + 1 - abar across them, so that
        C^-1 = U^T diag(1 / c_j) U + (I - U^T U) / c_perp.
    Score s_i(x) = -C^-1 (x - sqrt(abar) mu); its Jacobian -C^-1 is symmetric."""

    def __init__(self, mu, U, lam, s2: float):
        self.mu = np.asarray(mu, np.float64).ravel()
        self.U = np.asarray(U, np.float64).reshape(-1, self.mu.size)
        self.lam = np.asarray(lam, np.float64).ravel()
        self.s2 = float(s2)

    def _cinv(self, r, abar: float):
        """C^-1 r for r [B][n] (rows of U orthonormal)."""
        c = abar * (self.lam + self.s2) + 1.0 - abar
        cp = abar * self.s2 + 1.0 - abar
        p = r @ self.U.T                                     # [B][k]
        return (r - p @ self.U) / cp + (p / c) @ self.U

    def score(self, x, abar: float):
        x = np.asarray(x, np.float64)
        B = x.shape[0]
        r = x.reshape(B, -1) - np.sqrt(abar) * self.mu
        return -self._cinv(r, abar).reshape(x.shape)

    def score_vjp(self, g, abar: float):
        g = np.asarray(g, np.float64)
        B = g.shape[0]
        return -self._cinv(g.reshape(B, -1), abar).reshape(g.shape)


def clean_estimate(v_i, s, abar: float):
    """Eq. v0hat: (v_i + (1 - abar_i) s) / sqrt(abar_i)."""
    return (np.asarray(v_i, np.float64) + (1.0 - abar) * np.asarray(s, np.float64)) / np.sqrt(abar)


def proposal(v_i, v0hat, z, sched: Schedule, i: int):
    """The prior-driven proposal v'_{i-1} of Algorithms 1-2."""
    c_v, c_0, sg = sched.proposal_coefficients(i)
    return c_v * np.asarray(v_i, np.float64) + c_0 * np.asarray(v0hat, np.float64) + \
        sg * np.asarray(z, np.float64)


def to_physical(x0hat, shift=SHIFT, unit=UNIT, v_lo=V_LO, v_hi=V_HI):
    """(v = clamp(shift + unit x0hat, v_lo, v_hi), mask of the unclamped cells)."""
    v = shift + unit * np.asarray(x0hat, np.float64)
    mask = (v >= v_lo) & (v <= v_hi)
    return np.clip(v, v_lo, v_hi), mask


def guidance_gradients(g_phys, mask, abar: float, u=None, unit=UNIT):
    """g = dPhi/dx0hat (normalised) and h = dPhi/dv_i by Eq. chain_rule:
    x0hat = (v_i + (1 - abar) s(v_i)) / sqrt(abar), so
    h = (g + (1 - abar) (ds/dv_i)^T g) / sqrt(abar); ``u`` = (ds/dv_i)^T g
    (None: a score that does not depend on v_i)."""
    g = unit * np.asarray(g_phys, np.float64) * mask
    uu = 0.0 if u is None else np.asarray(u, np.float64)
    h = (g + (1.0 - abar) * uu) / np.sqrt(abar)
    return g, h


def w2_potential(prob: O.Problem, ctx: O.ObsContext, w2p: O.W2Params, threads=None):
    """Phi = J of Eq. final_objective: v [B][nz][nx] m/s -> (J [B], dJ/dv)."""

    def f(v):
        J, g, _ = O.gradient(prob, v, ctx, w2p, threads=threads)
        return J, g

    return f


def l2_potential(prob: O.Problem, d_obs, sigma: float):
    """Phi_l2 of Algorithm 1: (1/2) ||F(v) - d_obs||^2 / sigma^2 and its gradient."""
    d_obs = np.asarray(d_obs, np.float64)

    def f(v):
        v = np.asarray(v, np.float64)
        B = v.shape[0]
        J = np.zeros(B)
        g = np.zeros_like(v)
        for b in range(B):
            for s in range(prob.ns):
                d, u_all = O.forward_shot(prob, v[b], s, keep_wavefield=True)
                Jb, adj = O.l2_misfit(d_obs[b, s][None], d[None], sigma=sigma)
                J[b] += Jb[0]
                g[b] += O.fold(prob, O.adjoint_shot(prob, v[b], s, adj[0], u_all))
        return J, g

    return f


def reverse_step(sched: Schedule, i: int, v_i, z, potential, mu, tau2, gp: O.GuideParams,
                 dps_zeta: float | None = None, prior: LowRankPrior | None = None):
    """One reverse step i -> i-1 of Algorithm 2 (or, with ``dps_zeta``, of
    Algorithm 1: P_i = zeta I) for a batch v_i [B][nz][nx] in the normalised
    space, the Gaussian-prior score (``prior``: a LowRankPrior instead of
    mu, tau2) and a potential (``w2_potential`` or ``l2_potential``).
    Returns (v_{i-1}, a dict of the intermediates)."""
    abar = sched.abar[i]
    s = gaussian_score(v_i, abar, mu, tau2) if prior is None else prior.score(v_i, abar)
    x0 = clean_estimate(v_i, s, abar)
    vp = proposal(v_i, x0, z, sched, i)
    v_phys, mask = to_physical(x0)
    J, g_phys = potential(v_phys)
    g0, _ = guidance_gradients(g_phys, mask, abar)
    u = gaussian_score_vjp(g0, abar, tau2) if prior is None else prior.score_vjp(g0, abar)
    g, h = guidance_gradients(g_phys, mask, abar, u)
    if dps_zeta is not None:
        v_next = vp - dps_zeta * h
        rho = np.full(v_next.shape[0], dps_zeta)
    else:
        v_next, rho = O.guided_step(vp, x0, g, h, gp)
    return v_next, dict(score=s, v0hat=x0, v_prime=vp, v_phys=v_phys, mask=mask, J=J,
                        g_phys=g_phys, g=g, h=h, rho=rho)
