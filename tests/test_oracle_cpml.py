"""Pins of the CPML oracle (the PML reading of the paper's absorbing layer,
Sec. 6.1), CPU only:

* with sigma = 0 (refl_R = 1) the scheme is the undamped leapfrog of the
  sponge oracle, to rounding;
* the 4th-order first difference is exact on polynomials of degree <= 4 and
  antisymmetric (Dx^T = -Dx), the second difference symmetric, with zero
  values outside the grid (the GPU kernels use both identities);
* the adjoint solve passes the dot-product test against central differences
  of the forward;
* dJ/dv of the whole W2 objective matches central differences of J;
* the layer absorbs: energy left at the receivers after the direct and
  surface waves have passed is orders of magnitude below the sponge's and
  the reflecting edges' for the same layer width;
* the profiles vanish inside the physical grid and grow quadratically into
  the layer (b = exp(-sigma dt), a = b - 1).
"""
import dataclasses

import numpy as np
import pytest

from oracle import cpml as C
from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I


def _prob(nz=14, nx=16, nb=6, nt=150, ns=2, **kw):
    g = I.surface_geometry(nx, ns)
    base = dict(nz=nz, nx=nx, nb=nb, nt=nt, dz=10.0, dx=10.0, dt=1e-3, src_iz=g.src_iz,
                src_ix=g.src_ix, rec_iz=g.rec_iz, rec_ix=g.rec_ix, f_peak=40.0, v_ref=2500.0)
    base.update(kw)
    return O.Problem(**base)


def test_without_stretching_it_is_the_undamped_leapfrog():
    prob = _prob(refl_R=1.0)
    v = 1900 + 500 * np.random.default_rng(1).random((14, 16))
    for s in range(2):
        dc, ds = C.forward_shot(prob, v, s)[0], O.forward_shot(prob, v, s)[0]
        assert np.abs(dc - ds).max() <= 1e-12 * np.abs(ds).max()


@pytest.mark.parametrize("k", range(5))
def test_first_difference_exact_on_polynomials(k):
    prob = _prob(nz=9, nx=20, nb=0)
    Dx, Dz, _, _ = C.operators(prob)
    x = (np.arange(20) - 7) * prob.dx
    u = np.tile(x ** k, (9, 1))
    exact = np.tile(k * x ** max(k - 1, 0) if k else 0 * x, (9, 1))
    got = (Dx @ u.ravel()).reshape(9, 20)
    np.testing.assert_allclose(got[:, 2:-2], exact[:, 2:-2], rtol=1e-10,
                               atol=1e-10 * max(1.0, np.abs(exact).max()))
    z = (np.arange(9) - 4) * prob.dz
    uz = np.tile((z ** k)[:, None], (1, 20))
    gz = (Dz @ uz.ravel()).reshape(9, 20)
    ez = np.tile((k * z ** max(k - 1, 0) if k else 0 * z)[:, None], (1, 20))
    np.testing.assert_allclose(gz[2:-2], ez[2:-2], rtol=1e-10,
                               atol=1e-10 * max(1.0, np.abs(ez).max()))


def test_operator_symmetries():
    Dx, Dz, Dxx, Dzz = C.operators(_prob(nz=7, nx=9, nb=2))
    for D in (Dx, Dz):
        assert abs(D + D.T).max() == 0
    for D in (Dxx, Dzz):
        assert abs(D - D.T).max() == 0


def test_profiles():
    prob = _prob(nz=10, nx=12, nb=5)
    ax, bx, az, bz = C.profiles(prob)
    inner = np.s_[:10, 5:17]
    assert np.all(ax[inner] == 0) and np.all(bx[inner] == 1)
    assert np.all(az[:10] == 0)
    # sigma_x = d0 (d/nb)^2 in the d-th cell into the side layers
    d0 = 3 * prob.v_ref * np.log(1 / prob.refl_R) / (2 * prob.nb * prob.dx)
    for px, d in ((0, 5), (2, 3), (4, 1), (21, 5), (17, 1)):
        np.testing.assert_allclose(bx[3, px], np.exp(-d0 * (d / 5) ** 2 * prob.dt), rtol=1e-14)
        np.testing.assert_allclose(ax[3, px], bx[3, px] - 1, rtol=1e-14)
    np.testing.assert_allclose(bz[14, 8], np.exp(-d0 * (5 / 5) ** 2 * prob.dt), rtol=1e-14)


def test_adjoint_dot_product():
    prob = _prob()
    rng = np.random.default_rng(3)
    v = 1900 + 500 * rng.random((14, 16))
    dv = rng.standard_normal((14, 16))
    dd = rng.standard_normal((prob.nr, prob.nt))
    h = 1e-2
    dp = C.forward_shot(prob, v + h * dv, 1)[0]
    dm = C.forward_shot(prob, v - h * dv, 1)[0]
    lhs = np.vdot((dp - dm) / (2 * h), dd)
    _, rec = C.forward_shot(prob, v, 1, keep_record=True)
    rhs = np.vdot(dv, O.fold(prob, C.adjoint_shot(prob, v, 1, dd, rec)))
    assert abs(lhs - rhs) < 1e-7 * abs(rhs)


def test_gradient_matches_central_differences():
    prob = _prob(nz=12, nx=12, nb=4, nt=90)
    w2p = O.W2Params(n_xi=200)
    vt = 1800 + 400 * I.layered_model(1, 12, 12) / 4500.0 + I.smooth_perturbation(5, 12, 12, 150)
    v = 2000 + I.smooth_perturbation(6, 12, 12, 100)
    ctx = O.w2_prepare(C.forward(prob, vt[None]), prob.dt, w2p)
    J, g = C.gradient(prob, v[None], ctx, w2p)
    h = 1e-3
    for iz, ix in ((0, 0), (0, 5), (1, 11), (3, 3), (6, 8), (11, 0), (11, 11), (7, 1)):
        e = np.zeros_like(v)
        e[iz, ix] = h
        Jp = O.w2_misfit(ctx, C.forward(prob, (v + e)[None]), prob.dt, w2p, False)[0][0]
        Jm = O.w2_misfit(ctx, C.forward(prob, (v - e)[None]), prob.dt, w2p, False)[0][0]
        assert abs((Jp - Jm) / (2 * h) - g[0, iz, ix]) < 1e-5 * np.abs(g[0]).max()


def test_layer_absorbs_better_than_the_sponge():
    g = I.surface_geometry(40, 1)
    prob = O.Problem(nz=40, nx=40, nb=10, nt=700, dz=10.0, dx=10.0, dt=1e-3, src_iz=(20,),
                     src_ix=(20,), rec_iz=g.rec_iz, rec_ix=g.rec_ix, f_peak=25.0, v_ref=2500.0)
    v = np.full((40, 40), 2500.0)
    late = np.s_[:, 350:]                  # after the direct and surface-reflected waves
    e_cpml = (C.forward_shot(prob, v, 0)[0][late] ** 2).sum()
    e_sponge = (O.forward_shot(prob, v, 0)[0][late] ** 2).sum()
    e_refl = (O.forward_shot(dataclasses.replace(prob, refl_R=1.0), v, 0)[0][late] ** 2).sum()
    assert e_cpml < 1e-3 * e_sponge and e_sponge < 1e-2 * e_refl
