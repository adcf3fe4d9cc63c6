"""Pins of the oracle's preconditioned guided update (Sec. 5.2, Algorithm 2),
CPU only (P-11): closed forms of TV (Eq. tv), rho (Eq. rho), kappa (Eq. kappa)
and the reduction to the scalar DPS step when gamma = 0 (Eq. precond_step)."""
import numpy as np

from oracle import oracle as O


def _rand(seed, shape=(2, 9, 11)):
    return np.random.default_rng(seed).standard_normal(shape)


def test_constant_field_gives_rho0():
    v0 = np.full((1, 9, 11), 0.3)
    g, h, vp = _rand(1, v0.shape), _rand(2, v0.shape), _rand(3, v0.shape)
    gp = O.GuideParams(rho0=1.7, c=0.1, tau=0.0, gamma=0.0)
    vout, rho = O.guided_step(vp, v0, g, h, gp)
    assert rho[0] == 1.7
    np.testing.assert_allclose(vout, vp - 1.7 * h, rtol=1e-15)   # gamma = 0: kappa = 1


def test_linear_ramp_tv_closed_form():
    nz, nx, a, b = 9, 11, 0.03, -0.02
    iz, ix = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    v0 = (a * ix + b * iz)[None]
    tv = (abs(a) * (nx - 1) * nz + abs(b) * (nz - 1) * nx) / (nz * nx)
    z = np.zeros_like(v0)
    gp = O.GuideParams(rho0=2.0, c=0.1, tau=0.0, gamma=0.0)
    _, rho = O.guided_step(z, v0, z + 1, z, gp)
    np.testing.assert_allclose(rho[0], 2.0 * np.exp(-tv / 0.1), rtol=1e-14)
    # tau above TV switches the damping off; tau below shifts it
    _, rho = O.guided_step(z, v0, z + 1, z, O.GuideParams(rho0=2.0, c=0.1, tau=tv + 1e-3))
    assert rho[0] == 2.0
    _, rho = O.guided_step(z, v0, z + 1, z, O.GuideParams(rho0=2.0, c=0.1, tau=0.5 * tv))
    np.testing.assert_allclose(rho[0], 2.0 * np.exp(-0.5 * tv / 0.1), rtol=1e-14)


def test_kappa_properties():
    g = _rand(4)
    h = np.ones_like(g)
    z = np.zeros_like(g)
    gp = O.GuideParams(rho0=1.0, c=0.1, tau=0.0, gamma=0.55, eps=1e-4)
    vout, rho = O.guided_step(z, z, g, h, gp)
    kappa = -vout / rho[:, None, None]
    for b in range(g.shape[0]):
        gb = np.abs(g[b])
        assert np.all(kappa[b] >= 1 - 1e-15)
        assert abs(kappa[b].ravel()[np.argmax(gb)] - 1.0) < 1e-15
        # kappa is a decreasing function of |g|
        order = np.argsort(gb.ravel())
        assert np.all(np.diff(kappa[b].ravel()[order]) <= 1e-15)
        # closed form at the smallest |g|
        jmin = np.argmin(gb)
        np.testing.assert_allclose(kappa[b].ravel()[jmin],
                                   ((gb.max() + 1e-4) / (gb.ravel()[jmin] + 1e-4)) ** 0.55, rtol=1e-14)


def test_kappa_clipping():
    g = _rand(5)
    h = np.ones_like(g)
    z = np.zeros_like(g)
    gp = O.GuideParams(rho0=1.0, gamma=1.0, eps=1e-4, kappa_min=1.5, kappa_max=4.0)
    vout, _ = O.guided_step(z, z, g, h, gp)
    kappa = -vout
    assert kappa.min() >= 1.5 and kappa.max() <= 4.0
    assert np.any(kappa == 1.5) and np.any(kappa == 4.0)
