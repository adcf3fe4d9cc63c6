"""Pins of the oracle's wave solver (Eq. 1, Sec. 6.1), CPU only.

P-2 Ricker closed form; P-4 discrete energy conservation without damping and
decay with it; P-7 source/receiver reciprocity; P-8 mirror symmetry; P-10
agreement with the analytic 2D Green's function of Eq. (1) in a homogeneous
medium (which fixes the source scaling, the time alignment of the samples and
the velocity scaling).
"""
import numpy as np
import pytest

from oracle import oracle as O


def _prob(nz, nx, nb, nt, h=10.0, dt=1e-3, src=((0, 0),), rec=((0, 0),), **kw):
    return O.Problem(nz=nz, nx=nx, nb=nb, nt=nt, dz=h, dx=h, dt=dt,
                     src_iz=tuple(s[0] for s in src), src_ix=tuple(s[1] for s in src),
                     rec_iz=tuple(r[0] for r in rec), rec_ix=tuple(r[1] for r in rec), **kw)


def test_ricker_closed_form():
    fp = 15.0
    t0 = 1.1 / fp
    lib = O.lib()
    assert lib.orc_ricker(t0, fp, t0) == 1.0
    tz = 1 / (np.sqrt(2) * np.pi * fp)          # zeros of 1 - 2 a
    for t in (t0 - tz, t0 + tz):
        assert abs(lib.orc_ricker(t, fp, t0)) < 1e-15
    tm = np.sqrt(1.5) / (np.pi * fp)            # minima at a = 3/2
    for t in (t0 - tm, t0 + tm):
        np.testing.assert_allclose(lib.orc_ricker(t, fp, t0), -2 * np.exp(-1.5), rtol=1e-14)
        assert lib.orc_ricker(t + 1e-5, fp, t0) > lib.orc_ricker(t, fp, t0)
        assert lib.orc_ricker(t - 1e-5, fp, t0) > lib.orc_ricker(t, fp, t0)
    prob = _prob(4, 4, 0, 200)
    f = O.ricker_series(prob)
    np.testing.assert_allclose(f[73], lib.orc_ricker(0.073, 15.0, 1.1 / 15.0), rtol=1e-15)


def _energy(prob, v, u_all):
    """E^{n+1/2} = <(u^{n+1}-u^n)^2 / kappa> - <L u^{n+1}, u^n>: conserved by the
    undamped leapfrog with a symmetric L once the source is off."""
    kappa = (O.pad_model(prob, v) * prob.dt) ** 2
    E = []
    for n in range(prob.nt):
        du = u_all[n + 1] - u_all[n]
        Lu = O.laplacian(u_all[n + 1], prob.dz, prob.dx, 0)
        E.append(np.sum(du * du / kappa) - np.sum(Lu * u_all[n]))
    return np.array(E)


def test_energy_conserved_without_damping():
    nz, nx, nt = 30, 34, 400
    prob = _prob(nz, nx, 0, nt, src=((12, 15),), rec=((3, 3),), refl_R=1.0)
    rng = np.random.default_rng(0)
    v = 2000 + 600 * rng.random((nz, nx))
    f = O.ricker_series(O.Problem(**{**prob.__dict__, "f_peak": 25.0}))
    f[120:] = 0.0                                # source switched off exactly
    _, u_all = O.forward_shot(prob, v, 0, keep_wavefield=True, wavelet=f)
    E = _energy(prob, v, u_all)
    after = E[121:]
    assert after.min() > 0
    assert np.ptp(after) < 1e-11 * after.mean()
    assert np.abs(u_all[-1]).max() > 1e-3 * np.abs(u_all).max()  # wave still present


def test_energy_decays_with_absorbing_layer():
    nz, nx, nb, nt = 30, 34, 12, 600
    prob = _prob(nz, nx, nb, nt, src=((12, 15),), rec=((3, 3),), v_ref=2600.0, refl_R=1e-3)
    v = np.full((nz, nx), 2300.0)
    f = O.ricker_series(O.Problem(**{**prob.__dict__, "f_peak": 25.0}))
    f[120:] = 0.0
    _, u_all = O.forward_shot(prob, v, 0, keep_wavefield=True, wavelet=f)
    E = _energy(prob, v, u_all)
    after = E[121:]
    assert np.all(np.diff(after) <= 1e-12 * after[0])
    assert after[-1] < 0.05 * after[0]


def test_reciprocity_heterogeneous():
    # swap source and receiver cells: identical traces (injection and recording
    # are transposes of each other through kappa A, Sec. 2.1 restriction R)
    nz, nx, nb, nt = 24, 26, 8, 350
    rng = np.random.default_rng(3)
    v = 1800 + 1500 * rng.random((nz, nx))
    a, b = (2, 5), (17, 20)
    pa = _prob(nz, nx, nb, nt, src=(a,), rec=(b,), f_peak=20.0)
    pb = _prob(nz, nx, nb, nt, src=(b,), rec=(a,), f_peak=20.0)
    da = O.forward_shot(pa, v, 0)[0][0]
    db = O.forward_shot(pb, v, 0)[0][0]
    # kappa differs at a and b, but the recorded fields must still agree
    np.testing.assert_allclose(da, db, rtol=0, atol=1e-12 * np.abs(da).max())
    assert np.abs(da).max() > 0


def test_mirror_symmetry():
    nz, nx, nb, nt = 20, 21, 6, 300
    vz = np.linspace(1600, 3200, nz)
    v = np.repeat(vz[:, None], nx, axis=1)
    rec = tuple((0, r) for r in range(nx))
    prob = _prob(nz, nx, nb, nt, src=((0, 10),), rec=rec, f_peak=20.0)
    d = O.forward_shot(prob, v, 0)[0]
    np.testing.assert_allclose(d, d[::-1], rtol=0, atol=1e-13 * np.abs(d).max())
    # an asymmetric model breaks it
    v2 = v.copy()
    v2[5:9, 2:6] = 4000
    d2 = O.forward_shot(prob, v2, 0)[0]
    assert np.abs(d2 - d2[::-1]).max() > 1e-3 * np.abs(d2).max()


def _green2d(r, c, t, fp, t0, n=4000):
    """Analytic field of (1/c^2) u_tt - Lap u = f(t) delta(x) in 2D:
    u(r,t) = (1/2 pi) int_0^inf f(t - (r/c) cosh s) ds."""
    s = np.linspace(0.0, 8.0, n)
    tau = (r / c) * np.cosh(s)
    out = []
    for ti in t:
        a = np.pi ** 2 * fp ** 2 * (ti - tau - t0) ** 2
        out.append(np.trapezoid((1 - 2 * a) * np.exp(-a), s) / (2 * np.pi))
    return np.array(out)


def test_homogeneous_medium_matches_analytic_green_function():
    # fine grid, receiver in the interior, window closed before any boundary
    # reflection arrives
    h, dt, c, fp = 2.5, 2.5e-4, 2000.0, 25.0
    nz = nx = 161
    nt = 600
    src, rec = (80, 80), (80, 120)                 # offset 100 m
    prob = _prob(nz, nx, 20, nt, h=h, dt=dt, src=(src,), rec=(rec,), f_peak=fp,
                 v_ref=c, refl_R=1e-3)
    v = np.full((nz, nx), c)
    d = O.forward_shot(prob, v, 0)[0][0]
    # sample n is the field u^{n+1}, at time (n+1) dt
    t = (np.arange(nt) + 1) * dt
    g = _green2d(40 * h, c, t, fp, 1.1 / fp)
    err = np.linalg.norm(d - g) / np.linalg.norm(g)
    assert err < 3e-3, err
    # one sample of misalignment would be far outside that bound
    g_shift = _green2d(40 * h, c, t - dt, fp, 1.1 / fp)
    assert np.linalg.norm(d - g_shift) / np.linalg.norm(g) > 3 * err
