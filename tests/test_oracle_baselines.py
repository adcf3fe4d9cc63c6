"""Pins of the oracle's baseline potentials, TV subgradient and reconstruction
measures (Sec. 4.2, 6.3), CPU only.

* least squares (Baseline 3 potential): closed form for a constant residual,
  exact derivative;
* squared, unenhanced W2 (Baseline 1): per trace the square of the W2 the
  main objective uses, the translation closed form, central differences of
  the reverse pass (now also at W2 = 0, where the square is differentiable);
* TV of Eq. tv and its subgradient: closed forms on ramps, central
  differences away from ties, linearity in g and alpha;
* relative l2 error, PSNR, SSIM: closed forms for a constant offset,
  SSIM(x, x) = 1 and symmetry, an independent sliding-window evaluation.
"""
import numpy as np
import pytest

from oracle import oracle as O

DT = 1e-3


def gauss(mu, sig, nt=600, dt=DT):
    t = np.arange(nt) * dt
    return np.exp(-0.5 * ((t - mu) / sig) ** 2) / (sig * np.sqrt(2 * np.pi))


def _cube(seed, ns=2, nr=3, nt=400):
    rng = np.random.default_rng(seed)
    t = np.arange(nt) * DT
    d = np.zeros((1, ns, nr, nt))
    for s in range(ns):
        for r in range(nr):
            t0, f = rng.uniform(0.05, 0.3), rng.uniform(8, 25)
            a = np.pi ** 2 * f ** 2 * (t - t0) ** 2
            d[0, s, r] = rng.uniform(0.2, 1.0) * (1 - 2 * a) * np.exp(-a)
            d[0, s, r] += 0.01 * rng.standard_normal(nt)
    return d


# ---------------------------------------------------------------- least squares

def test_l2_closed_form_and_derivative():
    rng = np.random.default_rng(0)
    d_obs = rng.standard_normal((2, 3, 4, 50))
    J, adj = O.l2_misfit(d_obs, d_obs + 0.3, sigma=0.5)
    np.testing.assert_allclose(J, 0.5 * 0.09 / 0.25 * 600, rtol=1e-12)
    np.testing.assert_allclose(adj, 0.3 / 0.25, rtol=1e-12)
    d_syn = d_obs + rng.standard_normal(d_obs.shape)
    J, adj = O.l2_misfit(d_obs, d_syn, sigma=2.0)
    dd = rng.standard_normal(d_obs.shape)
    h = 1e-6
    fd = (O.l2_misfit(d_obs, d_syn + h * dd, 2.0)[0] - O.l2_misfit(d_obs, d_syn - h * dd, 2.0)[0]) / (2 * h)
    np.testing.assert_allclose(fd, (adj * dd).reshape(2, -1).sum(axis=1), rtol=1e-8)
    assert np.all(O.l2_misfit(d_obs, d_obs)[0] == 0)


# ---------------------------------------------------------------- squared W2

def test_squared_w2_is_the_square_of_the_trace_w2():
    d, syn = _cube(1), _cube(2)
    for k in (100.0, 0.0):
        base = O.W2Params(k=k, n_xi=300)
        sq = O.W2Params(k=k, n_xi=300, squared=True)
        ctx = O.w2_prepare(d, DT, base)
        _, w2, _ = O.w2_misfit(ctx, syn, DT, base, with_adjoint=False)
        J2, w2sq, _ = O.w2_misfit(ctx, syn, DT, sq, with_adjoint=False)
        np.testing.assert_allclose(w2sq, w2 ** 2, rtol=1e-13)
        np.testing.assert_allclose(ctx.S2, (ctx.s_tr ** 2).sum(axis=(1, 2)), rtol=1e-14)
        np.testing.assert_allclose(J2, (w2 ** 2).sum() / ctx.S2, rtol=1e-13)


def test_squared_w2_translation_closed_form():
    # one trace pair: translate a positive pulse by tau; W2^2 = tau^2 up to the
    # end nodes of the xi grid (whose quantiles clamp), and J = W2^2 / int Q_obs^2
    nxi = 2000
    a, b = gauss(0.20, 0.02), gauss(0.26, 0.02)
    w2p = O.W2Params(k=0.0, cshift_factor=0.0, n_xi=nxi, squared=True)
    ctx = O.w2_prepare(a[None, None, None], DT, w2p)
    J, w2sq, _ = O.w2_misfit(ctx, b[None, None, None], DT, w2p, with_adjoint=False)
    np.testing.assert_allclose(w2sq[0, 0, 0], 0.06 ** 2 * (nxi - 2) / (nxi - 1), rtol=2e-3)
    np.testing.assert_allclose(J[0], w2sq[0, 0, 0] / ctx.s_tr[0, 0, 0] ** 2, rtol=1e-13)


def test_squared_w2_adjoint_matches_central_differences():
    d, syn = _cube(3), _cube(4)
    w2p = O.W2Params(k=0.0, n_xi=400, squared=True)
    ctx = O.w2_prepare(d, DT, w2p)
    J, _, adj = O.w2_misfit(ctx, syn, DT, w2p)
    rng = np.random.default_rng(5)
    for _ in range(3):
        dd = rng.standard_normal(syn.shape)
        h = 1e-7
        fd = (O.w2_misfit(ctx, syn + h * dd, DT, w2p, False)[0][0] -
              O.w2_misfit(ctx, syn - h * dd, DT, w2p, False)[0][0]) / (2 * h)
        an = np.vdot(adj, dd)
        assert abs(fd - an) < 1e-6 * abs(an)
    # at the observation the square is differentiable with derivative 0
    _, _, adj0 = O.w2_misfit(ctx, d, DT, w2p)
    assert np.all(adj0 == 0)


# ---------------------------------------------------------------- TV subgradient

def test_tv_of_ramps_and_its_subgradient():
    nz, nx = 5, 7
    v = np.tile(3.0 * np.arange(nx), (nz, 1))[None]            # x ramp, slope 3
    tv, h = O.tv_grad(v, None, alpha=1.0, unit=1.5)
    np.testing.assert_allclose(tv[0], nz * (nx - 1) * 3.0 / 1.5 / (nz * nx), rtol=1e-14)
    # each x difference adds +1 to its right cell, -1 to its left cell
    expect = np.zeros((nz, nx))
    expect[:, 0], expect[:, -1] = -1.0, 1.0
    np.testing.assert_allclose(h[0], expect / (nz * nx * 1.5), rtol=1e-14)
    v = np.tile(-2.0 * np.arange(nz)[:, None], (1, nx))[None]  # decreasing z ramp
    tv, h = O.tv_grad(v, None, alpha=2.0, unit=1.0)
    np.testing.assert_allclose(tv[0], (nz - 1) * nx * 2.0 / (nz * nx), rtol=1e-14)
    expect = np.zeros((nz, nx))
    expect[0, :], expect[-1, :] = 1.0, -1.0
    np.testing.assert_allclose(h[0], 2.0 * expect / (nz * nx), rtol=1e-14)
    # ties (equal neighbours) contribute nothing
    tv, h = O.tv_grad(np.ones((1, 4, 4)), np.zeros((1, 4, 4)), alpha=5.0)
    assert tv[0] == 0 and np.all(h == 0)


def test_tv_subgradient_is_the_gradient_away_from_ties():
    rng = np.random.default_rng(7)
    v = rng.uniform(1500, 4500, (2, 9, 11))
    g = rng.standard_normal(v.shape)
    unit, alpha = 1500.0, 0.3
    tv, h = O.tv_grad(v, g, alpha, unit)
    dv = rng.standard_normal(v.shape)
    eps = 1e-2      # TV is piecewise linear: exact while no difference changes sign
    assert np.abs(np.diff(v, axis=2)).min() > 10 * eps and np.abs(np.diff(v, axis=1)).min() > 10 * eps
    tvp, _ = O.tv_grad(v + eps * dv, None, 1.0, unit)
    tvm, _ = O.tv_grad(v - eps * dv, None, 1.0, unit)
    fd = (tvp - tvm) / (2 * eps)
    np.testing.assert_allclose(alpha * fd, np.einsum("bij,bij->b", h - g, dv), rtol=1e-9)
    # linear in g and in alpha
    _, h2 = O.tv_grad(v, 2 * g, 2 * alpha, unit)
    np.testing.assert_allclose(h2, 2 * h, rtol=1e-13)


# ---------------------------------------------------------------- measures

def test_measures_closed_forms_for_an_offset():
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, (1, 30, 40))
    c, R = 0.05, 2.0
    m = O.image_metrics(x, x + c, R)[0]
    np.testing.assert_allclose(m[0], c * np.sqrt(x.size) / np.linalg.norm(x), rtol=1e-12)
    np.testing.assert_allclose(m[1], 10 * np.log10(R * R / c ** 2), rtol=1e-12)
    # an offset leaves variances and covariance unchanged: SSIM is the mean
    # over windows of the luminance term alone, with the window means of x
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    w2 = np.outer(w, w) / np.outer(w, w).sum()
    C1 = (0.01 * R) ** 2
    lum = []
    for i in range(30 - 10):
        for j in range(40 - 10):
            mu = (w2 * x[0, i:i + 11, j:j + 11]).sum()
            lum.append((2 * mu * (mu + c) + C1) / (mu ** 2 + (mu + c) ** 2 + C1))
    np.testing.assert_allclose(m[2], np.mean(lum), rtol=1e-12)


def test_ssim_identity_symmetry_and_sliding_windows():
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (1, 25, 33))
    y = x + 0.2 * rng.standard_normal(x.shape)
    assert O.image_metrics(x, x, 1.0)[0, 2] == pytest.approx(1.0, abs=1e-14)
    a, b = O.image_metrics(x, y, 1.0)[0, 2], O.image_metrics(y, x, 1.0)[0, 2]
    assert a == pytest.approx(b, rel=1e-14) and 0 < a < 1
    # independent evaluation: all windows at once, moments as E[x^2] - E[x]^2
    from numpy.lib.stride_tricks import sliding_window_view as swv
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    w2 = np.outer(w, w) / np.outer(w, w).sum()
    X, Y = swv(x[0], (11, 11)), swv(y[0], (11, 11))
    E = lambda A: np.einsum("ijab,ab->ij", A, w2)  # noqa: E731
    mx, my = E(X), E(Y)
    sxx, syy, sxy = E(X * X) - mx ** 2, E(Y * Y) - my ** 2, E(X * Y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = ((2 * mx * my + C1) * (2 * sxy + C2) / ((mx ** 2 + my ** 2 + C1) * (sxx + syy + C2))).mean()
    np.testing.assert_allclose(a, ssim, rtol=1e-10)
    # grids smaller than a window have no SSIM
    assert np.isnan(O.image_metrics(x[:, :10, :], y[:, :10, :], 1.0)[0, 2])
