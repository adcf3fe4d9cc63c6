"""Reverse-diffusion sampling with physics guidance on the library's kernels:
Algorithm 2 (OT-guided preconditioned DPS, Sec. 5.2) and Algorithm 1 (DPS
with the least-squares potential, Sec. 4.2).

One reverse step i -> i-1 for B states v_i [B][nz][nx] in the normalised
space x = (v - shift) / unit:
  1. the score s(v_i, i): a Gaussian prior (closed form, evaluated inside
     fwi_ddpm_proposal) or a caller's score model ``score_fn``;
  2. fwi_ddpm_proposal: v0hat (Eq. v0hat), the proposal v' and the clamped
     physical model v_phys in m/s;
  3. the potential's gradient at v_phys: J of Eq. final_objective
     (fwi_forward -> fwi_w2_misfit -> fwi_adjoint_grad) or Phi_l2; in the
     first reverse steps optionally the low-fidelity surrogate (LowFidelity);
  4. fwi_ddpm_guidance: g = dPhi/dv0hat and h = dPhi/dv_i (Eq. chain_rule);
  5. fwi_guided_step: v_{i-1} = v' - P_i h, P_i = rho_i D_i (Eq. precond_step),
     or P_i = zeta I (Algorithm 1).
Argument marshalling only: every step runs in the CUDA library (a caller's
``score_fn`` runs wherever the caller's model does).

A ``score_fn(v_i, i)`` returns ``(s, vjp)`` with ``s`` the score at v_i
([B][nz][nx] float32 on the device) and ``vjp(g)`` = (ds/dv_i)^T g.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Sequence

import numpy as np
import torch

from . import api

# P_i = zeta I through fwi_guided_step: gamma = 0 makes every kappa 1 and an
# unreachable TV threshold makes rho = rho0 = zeta
_TAU_NEVER = 1e30


def linear_betas(n: int, beta_1: float = 1e-4, beta_n: float = 0.02) -> list[float]:
    """beta_1..beta_N, linear from beta_1 to beta_N (the DDPM schedule; the
    paper fixes no values)."""
    return [float(b) for b in np.linspace(beta_1, beta_n, n)]


@dataclasses.dataclass
class GaussianPrior:
    """x_0 ~ N(mu, diag tau2) in the normalised space: a closed-form score
    model (the score of its step-i marginal, Eq. vp_transition).  ``mu`` and
    ``tau2`` are [nz][nx] float32 device tensors."""
    mu: torch.Tensor
    tau2: torch.Tensor

    @classmethod
    def from_models(cls, models, space: api.DiffusionSpace = api.DiffusionSpace(),
                    floor: float = 1e-3, device=None) -> "GaussianPrior":
        """Per-cell mean and variance of a set of velocity models [M][nz][nx]
        (m/s, host or device), mapped to the normalised space; the variance is
        kept >= ``floor``."""
        m = np.asarray(models.cpu() if torch.is_tensor(models) else models, dtype=np.float64)
        x = (m - space.shift) / space.unit
        mu = x.mean(axis=0)
        tau2 = np.maximum(x.var(axis=0), floor)
        dev = device or torch.device("cuda")
        return cls(torch.tensor(mu, dtype=torch.float32, device=dev),
                   torch.tensor(tau2, dtype=torch.float32, device=dev))


@dataclasses.dataclass
class LowRankPrior:
    """x_0 ~ N(mu, U^T diag(lam) U + s2 I) in the normalised space: the mean and
    the k leading principal directions of a set of models over an isotropic
    floor s2 (fwi_lowrank_score_at gives the score of its step-i marginal).
    Its samples are smooth where the diagonal prior's are rough cell by cell.
    ``mu`` [nz][nx], ``U`` [k][nz nx] (orthonormal rows), ``lam`` [k]: float32
    device tensors."""
    mu: torch.Tensor
    U: torch.Tensor
    lam: torch.Tensor
    s2: float

    @classmethod
    def from_models(cls, models, k: int = 32, space: api.DiffusionSpace = api.DiffusionSpace(),
                    floor: float = 1e-3, device=None) -> "LowRankPrior":
        """Principal components of velocity models [M][nz][nx] (m/s, host or
        device) in the normalised space: lam_j = S_j^2 / (M - 1) of the k
        largest singular values S_j of the centred models, s2 = the rest of the
        per-cell variance spread over the other directions, at least
        ``floor`` (fit on the host: set-up, not a step of the chain)."""
        m = np.asarray(models.cpu() if torch.is_tensor(models) else models, dtype=np.float64)
        M = m.shape[0]
        x = ((m - space.shift) / space.unit).reshape(M, -1)
        mu = x.mean(axis=0)
        _, S, Vt = np.linalg.svd(x - mu, full_matrices=False)
        k = min(k, Vt.shape[0])
        lam = S[:k] ** 2 / (M - 1)
        rest = float(np.sum(S[k:] ** 2) / (M - 1)) / max(x.shape[1] - k, 1)
        dev = device or torch.device("cuda")
        f32 = dict(dtype=torch.float32, device=dev)
        return cls(torch.tensor(mu.reshape(m.shape[1:]), **f32),
                   torch.tensor(np.ascontiguousarray(Vt[:k]), **f32),
                   torch.tensor(lam, **f32), max(rest, floor))


class LowFidelity:
    """The low-fidelity guidance surrogate (the multi-fidelity route to cheaper
    physics guidance, Sec. 7): the W2 potential of the problem coarsened by
    two in space and time (api.coarse_problem; about 8x fewer cell-updates),
    evaluated at R v with the observations decimated to the coarse
    acquisition, its gradient returned to the fine grid through R^T."""

    def __init__(self, plan: api.Plan, d_obs: torch.Tensor, w2: api.W2Params | None = None):
        self.fine = plan.prob
        self.plan = api.Plan(api.coarse_problem(plan.prob), w2 or plan.w2p, device=plan.device)
        self.ctx = self.plan.w2_prepare(api.fwi_decimate2(d_obs))

    def gradient(self, v_phys: torch.Tensor, stream=None, step: int = -1):
        """(J_c(R v) [B], R^T dJ_c/dv_c [B][nz][nx])."""
        vc = api.fwi_restrict2(v_phys, stream=stream)
        J, gc, _ = self.plan.gradient(vc, self.ctx, stream=stream)
        return J, api.fwi_restrict2_transpose(gc, self.fine.nz, self.fine.nx, stream=stream)


class NetworkSurrogate:
    """A learned surrogate of the physics guidance gradient (the surrogate
    route to cheaper guidance, Sec. 7): a convolutional network (ConvScore or
    UNetScore) trained on FD-generated pairs (v, dJ/dv) by
    DSMTrainer.regression_step, evaluated as
    dJ/dv ~ out_scale * net(in_scale * v, 0).  Its J is not available (None)."""

    def __init__(self, net, in_scale: float, out_scale: float):
        self.net, self.in_scale, self.out_scale = net, float(in_scale), float(out_scale)
        self.g = torch.empty(net.shape, dtype=torch.float32, device=net.dev)

    def gradient(self, v_phys: torch.Tensor, stream=None, step: int = -1):
        self.net.eps(v_phys, 0, self.out_scale, self.g, stream, in_scale=self.in_scale)
        return None, self.g


class Sampler:
    """Algorithm 2 (``guide`` = GuideParams) or Algorithm 1 (``dps_zeta``) on
    a plan of B models.

    potential: "w2" (J of Eq. final_objective; needs ``ctx`` from
    plan.w2_prepare), "l2" (Phi_l2 with ``d_obs`` and ``sigma_l2``) or None
    (no guidance: v_{i-1} = v').  Exactly one of ``prior`` and ``score_fn``.
    surrogate: a LowFidelity W2 potential, a NetworkSurrogate or a
    surrogate.GatedSurrogate (the learned forward surrogate checked by FD) used
    instead of the full one in the first ``surrogate_fraction`` of the reverse
    steps (i > N - round(fraction N)), the full physics after; its
    ``gradient(v_phys, stream=, step=)`` returns (J or None, dJ/dv)."""

    def __init__(self, plan: api.Plan, betas: Sequence[float], *, potential: str | None = "w2",
                 ctx=None, d_obs=None, sigma_l2: float = 1.0, prior: GaussianPrior | None = None,
                 score_fn: Callable | None = None, guide: api.GuideParams | None = None,
                 dps_zeta: float | None = None,
                 space: api.DiffusionSpace = api.DiffusionSpace(),
                 sigma_mode: int = api.SIGMA_POSTERIOR, surrogate: LowFidelity | None = None,
                 surrogate_fraction: float = 0.4):
        if (prior is None) == (score_fn is None):
            raise ValueError("give exactly one of prior and score_fn")
        if potential not in ("w2", "l2", None):
            raise ValueError(f"unknown potential {potential!r}")
        if potential == "w2" and ctx is None:
            raise ValueError("the W2 potential needs the observation context ctx")
        if potential == "l2" and d_obs is None:
            raise ValueError("the l2 potential needs d_obs")
        if potential is not None and (guide is None) == (dps_zeta is None):
            raise ValueError("give exactly one of guide (Algorithm 2) and dps_zeta (Algorithm 1)")
        if surrogate is not None and potential != "w2":
            raise ValueError("a surrogate stands in for the W2 potential")
        if not 0.0 <= surrogate_fraction <= 1.0:
            raise ValueError("surrogate_fraction must lie in [0, 1]")
        self.plan, self.potential, self.ctx, self.d_obs = plan, potential, ctx, d_obs
        self.sigma_l2, self.prior, self.score_fn, self.space = sigma_l2, prior, score_fn, space
        self.N = len(betas)
        self.surrogate = surrogate
        # reverse steps i > i_switch use the surrogate (the first fraction of them)
        self.i_switch = self.N - int(round(surrogate_fraction * self.N)) if surrogate else self.N
        self.steps = [None] + [api.fwi_ddpm_coefficients(betas, i, sigma_mode)
                               for i in range(1, self.N + 1)]
        if dps_zeta is not None:
            self.gparams = api.GuideParams(rho0=float(dps_zeta), c=1.0, tau=_TAU_NEVER,
                                           gamma=0.0, eps=1.0, unit=1.0)
        elif guide is not None:
            self.gparams = dataclasses.replace(guide, unit=1.0)
        else:
            self.gparams = None
        B, nz, nx = plan.model_shape
        self.B, self.ncell = B, nz * nx
        dev = plan.device
        new = lambda: torch.empty((B, nz, nx), dtype=torch.float32, device=dev)  # noqa: E731
        self.v0hat, self.v_prime, self.v_phys, self.g, self.h = (new() for _ in range(5))

    def uses_surrogate(self, i: int) -> bool:
        return self.surrogate is not None and i > self.i_switch

    def _physics_gradient(self, i, stream):
        if self.uses_surrogate(i):
            return self.surrogate.gradient(self.v_phys, stream=stream, step=i)
        if self.potential == "w2":
            J, g_phys, _ = self.plan.gradient(self.v_phys, self.ctx, stream=stream)
        else:
            d_syn, _ = self.plan.forward(self.v_phys, stream=stream)
            J, adj = self.plan.l2_misfit(self.d_obs, d_syn, self.sigma_l2, stream=stream)
            g_phys = self.plan.adjoint_grad(self.v_phys, adj, stream=stream)
        return J, g_phys

    def step(self, v_i: torch.Tensor, i: int, z: torch.Tensor, v_out: torch.Tensor | None = None,
             stream=None):
        """v_{i-1} from v_i and this step's standard normal draws z (both
        [B][nz][nx]).  Returns (v_{i-1}, {"J", "rho"}); J and rho are None
        without a potential."""
        if not 1 <= i <= self.N:
            raise ValueError(f"step {i} outside 1..{self.N}")
        st = self.steps[i]
        shape = (self.B,) + tuple(self.plan.model_shape[1:])
        api._f32(v_i, shape, "v_i")
        api._f32(z, shape, "z")
        if v_out is None:
            v_out = torch.empty_like(v_i)
        if self.prior is not None:
            score, vjp, mu, tau2 = None, None, self.prior.mu, self.prior.tau2
        else:
            score, vjp = self.score_fn(v_i, i)
            score = score.contiguous()
            api._f32(score, shape, "score")
            mu = tau2 = None
        api.fwi_ddpm_proposal(self.B, self.ncell, st, self.space, v_i, score, mu, tau2, z,
                              self.v0hat, self.v_prime, self.v_phys, stream)
        if self.potential is None:
            v_out.copy_(self.v_prime)
            return v_out, {"J": None, "rho": None}
        J, g_phys = self._physics_gradient(i, stream)
        if vjp is None:
            api.fwi_ddpm_guidance(self.B, self.ncell, st, self.space, self.v0hat, g_phys, None,
                                  tau2, self.g, self.h, stream)
        else:
            # the network's vjp needs g first: g (and h without the score
            # term), then h with (ds/dv_i)^T g
            api.fwi_ddpm_guidance(self.B, self.ncell, st, self.space, self.v0hat, g_phys, None,
                                  None, self.g, self.h, stream)
            u = vjp(self.g).contiguous()
            api._f32(u, shape, "vjp")
            api.fwi_ddpm_guidance(self.B, self.ncell, st, self.space, self.v0hat, g_phys, u,
                                  None, self.g, self.h, stream)
        v_out, rho = api.guided_step(self.v_prime, self.v0hat, self.g, self.h, self.gparams,
                                     v_out=v_out, stream=stream)
        return v_out, {"J": J, "rho": rho}

    def sample(self, v_start: torch.Tensor, noise: Callable[[int], torch.Tensor],
               i_start: int | None = None, i_stop: int = 1, stream=None) -> torch.Tensor:
        """Reverse steps i_start..i_stop (default N..1) from v_start; ``noise(i)``
        gives step i's draws z.  Returns the state after step i_stop."""
        v = v_start
        for i in range(i_start or self.N, i_stop - 1, -1):
            v, _ = self.step(v, i, noise(i), stream=stream)
        return v


class GraphChain:
    """Algorithm 2 with a Gaussian prior (diagonal, GaussianPrior, or low-rank,
    LowRankPrior: its score and the score's vector-Jacobian product from
    fwi_lowrank_score_at), one CUDA graph per kind of reverse
    step.  The step index lives in device memory (the step's last launch
    decrements it), the coefficients in a device table (api.ddpm_table) and the
    draws of every step in ``zs`` [N + 1][B][nz][nx] (row i for step i), so the
    launches of a reverse step -- proposal (fwi_ddpm_proposal_at), the guidance
    gradient, the chain rule (fwi_ddpm_guidance_at) and the preconditioned
    update written over the state -- are captured once per kind and replayed
    for every step of that kind:
      "fd"     the full W2 gradient (forward -> misfit -> adjoint)
      "sur"    a surrogate's gradient (surrogate.SurrogateGuidance)
      "check"  the full gradient drives the update, and the surrogate's
               gradient at the same model is compared with it: per-model
               relative L2 errors into ``err`` (the FD solver as the check)
    ``run`` replays the chain; with a surrogate, the steps i > i_switch (the
    first ``surrogate_fraction`` of the chain) run "check" every
    ``check_every`` steps and "sur" between checks until a check's largest
    error exceeds ``threshold``, then "fd" for the rest (FD as fallback)."""

    def __init__(self, plan: api.Plan, betas: Sequence[float], ctx,
                 prior: GaussianPrior | LowRankPrior,
                 guide: api.GuideParams, zs: torch.Tensor,
                 space: api.DiffusionSpace = api.DiffusionSpace(),
                 sigma_mode: int = api.SIGMA_POSTERIOR, surrogate=None,
                 surrogate_fraction: float = 0.4, threshold: float = 0.05,
                 check_every: int = 10):
        B, nz, nx = plan.model_shape
        self.N, self.B, self.ncell = len(betas), B, nz * nx
        if tuple(zs.shape) != (self.N + 1, B, nz, nx):
            raise ValueError(f"zs must be [{self.N + 1}][{B}][{nz}][{nx}]")
        self.plan, self.ctx, self.prior, self.zs = plan, ctx, prior, zs
        self.gparams = dataclasses.replace(guide, unit=1.0)
        dev = plan.device
        self.table = api.ddpm_table(list(betas), sigma_mode, space, dev)
        self.step = torch.full((1,), self.N, dtype=torch.int32, device=dev)
        new = lambda: torch.empty((B, nz, nx), dtype=torch.float32, device=dev)  # noqa: E731
        self.v, self.v0hat, self.v_prime, self.v_phys, self.g, self.h = (new() for _ in range(6))
        self.lowrank = isinstance(prior, LowRankPrior)
        if self.lowrank:
            self.score, self.u = new(), new()
            self.work = torch.empty(max(1, B * prior.U.shape[0]), dtype=torch.float32, device=dev)
        self.surrogate = surrogate
        self.i_switch = self.N - int(round(surrogate_fraction * self.N)) if surrogate else self.N
        self.threshold, self.check_every = float(threshold), int(check_every)
        self.err = torch.zeros(B, dtype=torch.float32, device=dev)
        self.graphs = {}
        self.records: list = []
        self.counts = {"fd": 0, "sur": 0, "check": 0}

    def _launches(self, kind: str, stream):
        B, n, N, P = self.B, self.ncell, self.N, self.prior
        if self.lowrank:
            api.fwi_lowrank_score_at(B, n, P.U, P.lam, P.s2, self.v, P.mu, self.table, self.step,
                                     N, self.work, self.score, stream)
            api.fwi_ddpm_proposal_at(B, n, self.table, self.step, N, self.v, self.score, None,
                                     None, self.zs, B * n, self.v0hat, self.v_prime, self.v_phys,
                                     stream)
        else:
            api.fwi_ddpm_proposal_at(B, n, self.table, self.step, N, self.v, None, P.mu, P.tau2,
                                     self.zs, B * n, self.v0hat, self.v_prime, self.v_phys,
                                     stream)
        if kind == "sur":
            _, g_phys = self.surrogate.gradient(self.v_phys, stream=stream)
        else:
            _, g_phys, _ = self.plan.gradient(self.v_phys, self.ctx, stream=stream)
            if kind == "check":
                _, g_sur = self.surrogate.gradient(self.v_phys, stream=stream)
                api.fwi_rel_error(g_sur, g_phys, self.err, stream)
        if self.lowrank:
            # g first, then the score's vector-Jacobian product of g, then h
            api.fwi_ddpm_guidance_at(B, n, self.table, self.step, N, self.v0hat, g_phys, None,
                                     None, self.g, self.h, stream)
            api.fwi_lowrank_score_at(B, n, P.U, P.lam, P.s2, self.g, None, self.table,
                                     self.step, N, self.work, self.u, stream)
            api.fwi_ddpm_guidance_at(B, n, self.table, self.step, N, self.v0hat, g_phys, self.u,
                                     None, self.g, self.h, stream)
        else:
            api.fwi_ddpm_guidance_at(B, n, self.table, self.step, N, self.v0hat, g_phys, None,
                                     P.tau2, self.g, self.h, stream)
        api.guided_step(self.v_prime, self.v0hat, self.g, self.h, self.gparams, v_out=self.v,
                        stream=stream)
        api.fwi_ddpm_step_down(self.step, stream)

    def capture(self, kind: str):
        """Capture one reverse step of ``kind`` (the state and step index are
        restored after the untimed warm-up launches)."""
        if kind != "fd" and self.surrogate is None:
            raise ValueError(f"step kind {kind!r} needs a surrogate")
        v0, s0 = self.v.clone(), self.step.clone()
        cur = torch.cuda.current_stream(self.plan.device)
        side = torch.cuda.Stream(device=self.plan.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            self._launches(kind, side)
        cur.wait_stream(side)
        self.v.copy_(v0)
        self.step.copy_(s0)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._launches(kind, torch.cuda.current_stream(self.plan.device))
        self.graphs[kind] = graph
        self.v.copy_(v0)
        self.step.copy_(s0)
        return graph

    def run(self, v_start: torch.Tensor, i_start: int | None = None, i_stop: int = 1):
        """Reverse steps i_start..i_stop (default N..1) from v_start by graph
        replays; returns the state after step i_stop (self.v)."""
        i_start = i_start or self.N
        for k in (["fd"] + (["sur", "check"] if self.surrogate is not None else [])):
            if k not in self.graphs:
                self.capture(k)
        self.v.copy_(v_start)
        self.step.fill_(i_start)
        rejected, since = False, None
        for i in range(i_start, i_stop - 1, -1):
            if i > self.i_switch and not rejected:
                if since is None or since >= self.check_every:
                    self.graphs["check"].replay()
                    err = float(self.err.max())           # the FD check's verdict (a host read)
                    rejected = err > self.threshold
                    self.records.append((i, err, not rejected))
                    self.counts["check"] += 1
                    since = 1
                    continue
                self.graphs["sur"].replay()
                self.counts["sur"] += 1
                since += 1
            else:
                self.graphs["fd"].replay()
                self.counts["fd"] += 1
        return self.v
