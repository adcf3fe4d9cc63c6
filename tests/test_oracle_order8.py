"""Pins of the oracle's 8th-order variant (the space order of the paper's
solver, Sec. 6.1; reading C-1 keeps 4th order for the hot path), CPU only.

* the Laplacian is exact on polynomials of degree <= 9 and its error on x^10
  is -(h^8 / 3150) 10! = -1152 h^8 (the stencil's truncation term);
* the mirrored top (u[-k] = u[k], k = 1..4) is exact for even functions;
* <L u, w> = <u, L^T w> for both top boundaries;
* the undamped leapfrog conserves the discrete energy;
* the wave adjoint passes the dot-product test and dJ/dv matches central
  differences of the full objective (both top boundaries).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I


@pytest.mark.parametrize("k", range(10))
def test_exact_on_polynomials_up_to_degree_9(k):
    h = 0.37
    x = (np.arange(30) - 12) * h
    u = np.tile(x ** k, (20, 1))
    lap = O.laplacian(u, dz=h, dx=h, order=8)
    exact = k * (k - 1) * x ** max(k - 2, 0) if k >= 2 else 0 * x
    np.testing.assert_allclose(lap[5:15, 4:-4], np.tile(exact, (20, 1))[5:15, 4:-4],
                               rtol=1e-9, atol=1e-9 * max(1.0, np.abs(exact).max()))
    uz = u.T.copy()
    lapz = O.laplacian(uz, dz=h, dx=2 * h, order=8)
    np.testing.assert_allclose(lapz[4:-4, 5:15], np.tile(exact, (20, 1)).T[4:-4, 5:15],
                               rtol=1e-9, atol=1e-9 * max(1.0, np.abs(exact).max()))


def test_tenth_degree_truncation_term():
    h = 0.5
    x = (np.arange(24) - 11) * h
    u = np.tile(x ** 10, (16, 1))
    lap = O.laplacian(u, dz=1.0, dx=h, order=8)[6:10, 4:-4]
    exact = 90 * x[4:-4] ** 8
    np.testing.assert_allclose(lap - exact, -1152.0 * h ** 8, rtol=1e-7)


def test_mirror_top_is_exact_for_even_functions():
    h = 0.3
    z = np.arange(20) * h
    for p in (2, 4, 6, 8):
        u = np.tile((z ** p)[:, None], (1, 18))
        lap = O.laplacian(u, dz=h, dx=h, top_bc=1, order=8)
        np.testing.assert_allclose(lap[:6, 4:-4], p * (p - 1) * np.tile(z[:6, None] ** (p - 2), (1, 10)),
                                   rtol=1e-9, atol=1e-8)


@pytest.mark.parametrize("top_bc", [0, 1])
def test_transpose_identity(top_bc):
    rng = np.random.default_rng(4)
    u, w = rng.standard_normal((2, 17, 23))
    Lu = O.laplacian(u, 0.7, 1.3, top_bc, order=8)
    LTw = O.laplacian(w, 0.7, 1.3, top_bc, transpose=True, order=8)
    assert abs(np.vdot(Lu, w) - np.vdot(u, LTw)) < 1e-12 * np.abs(Lu).sum()


def test_energy_conserved_without_damping():
    nz, nx, nt = 30, 34, 400
    prob = O.Problem(nz=nz, nx=nx, nb=0, nt=nt, dz=10.0, dx=10.0, dt=1e-3, src_iz=(12,),
                     src_ix=(15,), rec_iz=(3,), rec_ix=(3,), f_peak=25.0, refl_R=1.0,
                     space_order=8)
    rng = np.random.default_rng(0)
    v = 2000 + 600 * rng.random((nz, nx))
    f = O.ricker_series(prob)
    f[120:] = 0.0
    _, u_all = O.forward_shot(prob, v, 0, keep_wavefield=True, wavelet=f)
    kappa = (O.pad_model(prob, v) * prob.dt) ** 2
    E = []
    for n in range(121, nt):
        du = u_all[n + 1] - u_all[n]
        Lu = O.laplacian(u_all[n + 1], prob.dz, prob.dx, 0, order=8)
        E.append(np.sum(du * du / kappa) - np.sum(Lu * u_all[n]))
    E = np.array(E)
    assert E.min() > 0 and np.ptp(E) < 1e-11 * E.mean()


def _tiny(top_bc, nz=12, nx=12, nb=4, nt=90, ns=2):
    g = I.surface_geometry(nx, ns)
    return O.Problem(nz=nz, nx=nx, nb=nb, nt=nt, dz=10.0, dx=10.0, dt=1e-3, src_iz=g.src_iz,
                     src_ix=g.src_ix, rec_iz=g.rec_iz, rec_ix=g.rec_ix, f_peak=40.0,
                     v_ref=2500.0, top_bc=top_bc, space_order=8)


@pytest.mark.parametrize("top_bc", [0, 1])
def test_wave_adjoint_dot_product(top_bc):
    prob = _tiny(top_bc, nz=10, nx=14, nb=5, nt=120, ns=1)
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


@pytest.mark.parametrize("top_bc", [0, 1])
def test_gradient_matches_central_differences(top_bc):
    prob = _tiny(top_bc)
    w2p = O.W2Params(n_xi=200)
    vt = 1800 + 400 * I.layered_model(1, 12, 12) / 4500.0 + I.smooth_perturbation(5, 12, 12, 150)
    v = 2000 + I.smooth_perturbation(6, 12, 12, 100)
    ctx = O.w2_prepare(O.forward(prob, vt[None]), prob.dt, w2p)
    J, g, _ = O.gradient(prob, v[None], ctx, w2p)
    h = 1e-3
    for iz, ix in ((0, 0), (0, 5), (1, 11), (3, 3), (6, 8), (11, 0), (11, 11), (7, 1)):
        e = np.zeros_like(v)
        e[iz, ix] = h
        Jp = O.w2_misfit(ctx, O.forward(prob, (v + e)[None], threads=1), prob.dt, w2p, False)[0][0]
        Jm = O.w2_misfit(ctx, O.forward(prob, (v - e)[None], threads=1), prob.dt, w2p, False)[0][0]
        assert abs((Jp - Jm) / (2 * h) - g[0, iz, ix]) < 1e-5 * np.abs(g[0]).max()
