"""Drivers of the paper's comparison methods that run on the library's hot
path (Sec. 4.2, 6.3).  Only loop control lives here; every step is a call
of the C ABI (forward, misfit, adjoint, TV subgradient, guided update).

  w2_tv_descent   Baseline 1 (W2 + TV): (sub)gradient descent on
                  sum W2^2 / sum |Q_obs|^2 (unenhanced: k = 0) + alpha TV with
                  a fixed step rho0,
                      v_n <- v_n - rho0 (grad_{v_n} J_raw + alpha g_TV(v_n))
  ot_we_tv_descent Baseline 2 (OT-WE + TV): the enhanced objective J of
                  Eq. final_objective + alpha TV, diagonal preconditioned step
                      v <- v - rho(v) D(v) (grad J + alpha g_TV)
                  with rho of Eq. rho and D of Eq. kappa evaluated at v
  l2_gradient     the least-squares potential of the DPS baseline and its
                  gradient, Phi_l2 = (1/2) ||F(v) - y||^2 / sigma^2

Steps are taken in the normalised space v_n = v / unit of the diffusion
prior (the guided update's convention): in physical units the descent step
is v <- v - rho0 unit^2 h with h = grad_v J + alpha dTV(v / unit)/dv.
"""
from __future__ import annotations

import dataclasses

import torch

from . import api


def w2_tv_params() -> api.W2Params:
    """Misfit parameters of Baseline 1: no wavefield enhancement (k = 0),
    squared W2 normalised by sum |Q_obs|^2."""
    return api.W2Params(k=0.0, squared=True)


def _descend(plan, ctx, v, alpha, gparams, iters, stream=None):
    history = []
    for _ in range(iters):
        J, g, _ = plan.gradient(v, ctx, stream=stream)
        h, tv = api.tv_grad(v, g, alpha, gparams.unit, stream=stream)
        v, rho = api.guided_step(v, v, g, h, gparams, stream=stream)
        history.append((J, tv, rho))
    return v, history


def w2_tv_descent(plan, ctx, v, alpha: float, rho0: float, iters: int, unit: float = 1500.0,
                  stream=None):
    """Baseline 1.  ``plan`` must carry ``w2_tv_params()`` and ``ctx`` its
    prepared observations.  Returns (v, [(J, TV, rho) per iteration])."""
    if not (plan.w2p.squared and plan.w2p.k == 0.0):
        raise ValueError("Baseline 1 needs the squared, unenhanced misfit (w2_tv_params())")
    # gamma = 0 makes D = I, an unreachable threshold tau keeps rho = rho0
    gparams = api.GuideParams(rho0=rho0, c=1.0, tau=3.0e38, gamma=0.0, unit=unit)
    return _descend(plan, ctx, v, alpha, gparams, iters, stream)


def ot_we_tv_descent(plan, ctx, v, alpha: float, gparams: api.GuideParams, iters: int,
                     stream=None):
    """Baseline 2 with P(v) = rho(v) D(v) from ``gparams`` (Eq. rho, Eq. kappa
    at v).  Returns (v, [(J, TV, rho) per iteration])."""
    return _descend(plan, ctx, v, alpha, dataclasses.replace(gparams), iters, stream)


def l2_gradient(plan, v, d_obs, sigma: float = 1.0, stream=None):
    """(Phi_l2 [B], dPhi_l2/dv [B][nz][nx]) of the DPS baseline's potential."""
    d_syn, _ = plan.forward(v, stream=stream)
    J, adj = plan.l2_misfit(d_obs, d_syn, sigma, stream=stream)
    grad = plan.adjoint_grad(v, adj, stream=stream)
    return J, grad
