"""Pins of the oracle's gradient dJ/dv (discrete adjoint, Sec. 4.2 F'*,
Sec. 5.2 "automatic differentiation"), CPU only.

P-5: brute force -- central differences of the full J on a tiny grid for every
cell; P-6: dot-product tests of the wave adjoint; P-12: a small preconditioned
step decreases J (descent lemma, Sec. 5.2).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I


def tiny_problem(top_bc=0, nz=12, nx=12, nb=4, nt=90, ns=2):
    g = I.surface_geometry(nx, ns)
    return O.Problem(nz=nz, nx=nx, nb=nb, nt=nt, dz=10.0, dx=10.0, dt=1e-3,
                     src_iz=g.src_iz, src_ix=g.src_ix, rec_iz=g.rec_iz, rec_ix=g.rec_ix,
                     f_peak=40.0, v_ref=2500.0, top_bc=top_bc)


def J_of(prob, v, ctx, w2p):
    d = O.forward(prob, v[None], threads=1)
    return O.w2_misfit(ctx, d, prob.dt, w2p, with_adjoint=False)[0][0]


@pytest.mark.parametrize("top_bc", [0, 1])
def test_gradient_matches_central_differences_every_cell(top_bc):
    prob = tiny_problem(top_bc)
    w2p = O.W2Params(n_xi=200)
    vt = 1800 + 400 * I.layered_model(1, 12, 12) / 4500.0 + I.smooth_perturbation(5, 12, 12, 150)
    v = 2000 + I.smooth_perturbation(6, 12, 12, 100)
    dobs = O.forward(prob, vt[None])
    ctx = O.w2_prepare(dobs, prob.dt, w2p)
    J, g, _ = O.gradient(prob, v[None], ctx, w2p)
    assert J[0] > 0
    h = 1e-3
    fd = np.zeros_like(v)
    for iz in range(12):
        for ix in range(12):
            e = np.zeros_like(v)
            e[iz, ix] = h
            fd[iz, ix] = (J_of(prob, v + e, ctx, w2p) - J_of(prob, v - e, ctx, w2p)) / (2 * h)
    rel = np.linalg.norm(fd - g[0]) / np.linalg.norm(fd)
    assert rel < 1e-6, rel
    assert np.max(np.abs(fd - g[0])) < 1e-5 * np.abs(fd).max()


@pytest.mark.parametrize("top_bc", [0, 1])
def test_wave_adjoint_dot_product(top_bc):
    # <F'(v) dv, dd> = <dv, F'(v)^T dd>, F' by central differences in FP64
    prob = tiny_problem(top_bc, nz=10, nx=14, nb=5, nt=120, ns=1)
    rng = np.random.default_rng(3)
    v = 1900 + 500 * rng.random((10, 14))
    dv = rng.standard_normal((10, 14))
    dd = rng.standard_normal((prob.nr, prob.nt))
    h = 1e-2
    dp = O.forward_shot(prob, v + h * dv, 0)[0]
    dm = O.forward_shot(prob, v - h * dv, 0)[0]
    lhs = np.vdot((dp - dm) / (2 * h), dd)
    _, u_all = O.forward_shot(prob, v, 0, keep_wavefield=True)
    rhs = np.vdot(dv, O.fold(prob, O.adjoint_shot(prob, v, 0, dd, u_all)))
    assert abs(lhs - rhs) < 1e-8 * abs(rhs)


def test_pipeline_pieces_agree():
    # gradient() = forward -> w2_misfit -> adjoint_shot -> fold, shot by shot
    prob = tiny_problem(nt=80)
    w2p = O.W2Params(n_xi=150)
    vt = I.layered_model(2, 12, 12) * 0.5 + 800
    v = I.linear_initial_model(12, 12) * 0.5 + 800
    ctx = O.w2_prepare(O.forward(prob, vt[None]), prob.dt, w2p)
    J, g, w2 = O.gradient(prob, v[None], ctx, w2p)
    d = O.forward(prob, v[None])
    J2, w22, adj = O.w2_misfit(ctx, d, prob.dt, w2p)
    g2 = np.zeros((12, 12))
    for s in range(prob.ns):
        _, u_all = O.forward_shot(prob, v, s, keep_wavefield=True)
        g2 += O.fold(prob, O.adjoint_shot(prob, v, s, adj[0, s], u_all))
    np.testing.assert_allclose(J, J2, rtol=1e-13)
    np.testing.assert_allclose(w2, w22, rtol=1e-13)
    np.testing.assert_allclose(g[0], g2, rtol=1e-12, atol=1e-12 * np.abs(g2).max())


def test_preconditioned_step_decreases_misfit():
    # descent lemma (Eq. descent_lemma): a small step along -rho D grad J lowers J
    prob = tiny_problem(nz=14, nx=16, nb=5, nt=110, ns=3)
    w2p = O.W2Params(n_xi=200)
    vt = I.layered_model(4, 14, 16) * 0.4 + 1000
    v = I.linear_initial_model(14, 16) * 0.4 + 1000
    ctx = O.w2_prepare(O.forward(prob, vt[None]), prob.dt, w2p)
    J0, g, _ = O.gradient(prob, v[None], ctx, w2p)
    gp = O.GuideParams(rho0=1.0, gamma=0.5, c=0.1, tau=0.0)
    # TV is taken on the normalised field (v - 3000)/1500 (reading C-13)
    vn = (v[None] - 3000.0) / 1500.0
    vout, rho = O.guided_step(v[None], vn, g, g, gp)
    assert 0 < rho[0] < 1
    upd = v[None] - vout
    # step size chosen so that max |update| is 2 m/s
    scale = 2.0 / np.abs(upd).max()
    v1 = v - scale * upd[0]
    J1 = J_of(prob, v1, ctx, w2p)
    assert J1 < J0[0]
    # and the first-order prediction holds: J1 - J0 ~ -<g, step>
    pred = -np.vdot(g[0], scale * upd[0])
    assert abs((J1 - J0[0]) - pred) < 0.1 * abs(pred)
