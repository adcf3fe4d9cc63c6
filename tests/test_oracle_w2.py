"""Pins of the oracle's W2 misfit (Sec. 5.1, 6.2), CPU only.

P-3: closed forms of the 1D quadratic Wasserstein distance through quantile
functions (Eq. Wp_1d): translation, Gaussians, and the library inverse of a
monotone piecewise-linear CDF.  The CDF is checked against scipy's cumulative
trapezoid.  P-9: J(d_obs) = 0, k = 0 gives omega = 1, invariance under a
common rescaling.  The hand-written reverse pass is checked against central
differences of the forward pass.
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O

DT = 1e-3
NT = 1000
NXI = 1000


def gauss(mu, sig, nt=NT, dt=DT):
    t = np.arange(nt) * dt
    return np.exp(-0.5 * ((t - mu) / sig) ** 2) / (sig * np.sqrt(2 * np.pi))


def test_cdf_is_cumulative_trapezoid():
    rng = np.random.default_rng(0)
    y = rng.uniform(0.1, 2.0, NT)
    p, F, Z = O.cdf(y, DT, 1e-9)
    np.testing.assert_allclose(Z, integrate.trapezoid(y, dx=DT), rtol=1e-13)
    np.testing.assert_allclose(p, y / (Z + 1e-9), rtol=1e-14)
    np.testing.assert_allclose(F, integrate.cumulative_trapezoid(p, dx=DT, initial=0), rtol=1e-12,
                               atol=1e-15)


def test_quantiles_are_the_inverse_of_the_linear_interpolant():
    # monotone CDF with flat parts: np.interp on (F, t) is the inverse except on
    # flat pieces, where the generalised inverse takes the left end
    rng = np.random.default_rng(1)
    p = rng.uniform(0.0, 1.0, NT)
    p[200:260] = 0.0
    p /= integrate.trapezoid(p, dx=DT) * (1 + 1e-6)
    F = integrate.cumulative_trapezoid(p, dx=DT, initial=0)
    t = np.arange(NT) * DT
    Q, ks = O.quantiles(F, DT, NXI)
    xi = np.arange(NXI) / (NXI - 1)
    inside = (xi > 0) & (xi <= F[-1])
    # strictly increasing part of F for the library inverse
    keep = np.concatenate([[True], np.diff(F) > 0])
    ref = np.interp(xi[inside], F[keep], t[keep])
    np.testing.assert_allclose(Q[inside], ref, rtol=0, atol=1e-12)
    assert Q[0] == 0.0 and Q[-1] == t[-1]          # clamped ends
    assert np.all(ks[~inside & (xi > 0)] == NT)


def test_quantiles_brute_force_nonmonotone():
    # a CDF that decreases in places (negative density, reading C-16): compare
    # with min{k : F_k >= xi} found by a plain scan for every xi
    rng = np.random.default_rng(2)
    F = np.cumsum(rng.normal(0.002, 0.004, 300))
    F[0] = 0.0
    Q, ks = O.quantiles(F, DT, 257)
    for j in range(257):
        xi = j / 256
        k = next((k for k in range(300) if F[k] >= xi), 300)
        assert ks[j] == k
        if k == 0:
            q = 0.0
        elif k == 300:
            q = 299 * DT
        else:
            q = (k - 1) * DT + DT * (xi - F[k - 1]) / (F[k] - F[k - 1])
        assert abs(Q[j] - q) <= 1e-15


def test_w2_translation_is_the_shift():
    # an exact shift by m samples moves every interior quantile by m dt; the two
    # clamped end nodes (xi = 0 and xi = 1) contribute nothing
    m = 100
    ya = gauss(0.40, 0.03)
    yb = np.concatenate([np.zeros(m), ya[:-m]])
    w = O.w2_signals(ya, yb, DT)
    expect = m * DT * np.sqrt((NXI - 2) / (NXI - 1))
    assert abs(w - expect) < 1e-9 * expect
    assert O.w2_signals(ya, ya, DT) == 0.0
    assert w == O.w2_signals(yb, ya, DT)


@pytest.mark.parametrize("mu2,s2", [(0.45, 0.03), (0.40, 0.05), (0.55, 0.02)])
def test_w2_gaussians(mu2, s2):
    mu1, s1 = 0.40, 0.03
    ya, yb = gauss(mu1, s1), gauss(mu2, s2)
    w = O.w2_signals(ya, yb, DT)
    # continuum closed form W2^2 = (mu1-mu2)^2 + (s1-s2)^2; the discrete rule
    # clamps the two end nodes, which removes the O(dxi log(1/dxi)) tails
    cont = np.sqrt((mu1 - mu2) ** 2 + (s1 - s2) ** 2)
    assert abs(w - cont) < 0.02 * cont
    # discrete expectation: exact Gaussian quantiles at the interior nodes,
    # trapezoid in xi; differs from the oracle only by the O(dt^2) CDF error
    xi = np.arange(1, NXI - 1) / (NXI - 1)
    dq = (mu1 - mu2) + (s1 - s2) * special.ndtri(xi)
    disc = np.sqrt(np.sum(dq ** 2) / (NXI - 1))
    assert abs(w - disc) < 2e-4 * disc


def _cube(seed, ns=2, nr=3, nt=400, scale=1.0):
    rng = np.random.default_rng(seed)
    t = np.arange(nt) * DT
    d = np.zeros((1, ns, nr, nt))
    for s in range(ns):
        for r in range(nr):
            t0 = rng.uniform(0.05, 0.3)
            f = rng.uniform(8, 25)
            a = np.pi ** 2 * f ** 2 * (t - t0) ** 2
            d[0, s, r] = scale * rng.uniform(0.2, 1.0) * (1 - 2 * a) * np.exp(-a)
            d[0, s, r] += 0.01 * scale * rng.standard_normal(nt)
    return d


def test_prepare_closed_forms():
    d = _cube(3)
    w2p = O.W2Params(n_xi=500)
    ctx = O.w2_prepare(d, DT, w2p)
    M = np.abs(d).max()
    assert ctx.M[0] == M
    np.testing.assert_allclose(ctx.omega, 1 / (1 + 100 * np.abs(d) / M), rtol=1e-15)
    mins = np.min(ctx.omega * d, axis=-1)
    np.testing.assert_allclose(ctx.cshift, 1.1 * np.abs(mins), rtol=1e-15)
    np.testing.assert_allclose(ctx.S_obs[0], ctx.s_tr.sum(), rtol=1e-14)
    # k = 0: omega == 1 (Eq. omega_def)
    ctx0 = O.w2_prepare(d, DT, O.W2Params(k=0.0, n_xi=500))
    assert np.all(ctx0.omega == 1.0)


def test_prepare_scale_of_a_uniform_trace():
    # a constant trace maps to the uniform density on [0, T]; its quantile is
    # xi T (T = (nt-1) dt) and (int_0^1 (xi T)^2)^(1/2) = T / sqrt(3) up to the
    # trapezoid error of xi^2 (dxi^2 / 6) and eps'
    nt, nxi = 400, 500
    d = np.ones((1, 1, 1, nt))
    ctx = O.w2_prepare(d, DT, O.W2Params(k=0.0, n_xi=nxi))
    T = (nt - 1) * DT
    dxi = 1 / (nxi - 1)
    np.testing.assert_allclose(ctx.s_tr[0, 0, 0], T * np.sqrt(1 / 3 + dxi ** 2 / 6), rtol=1e-6)


def test_misfit_zero_at_observation_and_scale_invariance():
    d = _cube(4)
    w2p = O.W2Params(n_xi=500)
    ctx = O.w2_prepare(d, DT, w2p)
    J, w2, adj = O.w2_misfit(ctx, d, DT, w2p)
    assert J[0] == 0.0 and np.all(w2 == 0) and np.all(adj == 0)
    syn = _cube(5)
    J1 = O.w2_misfit(ctx, syn, DT, w2p, with_adjoint=False)[0]
    # common rescaling of obs and syn: omega, the density and the quantiles are
    # unchanged up to eps' (Sec. 6.2)
    ctx2 = O.w2_prepare(7.0 * d, DT, w2p)
    J2 = O.w2_misfit(ctx2, 7.0 * syn, DT, w2p, with_adjoint=False)[0]
    np.testing.assert_allclose(J2, J1, rtol=1e-6)
    assert J1[0] > 0


def test_misfit_is_normalised_sum_of_w2():
    d, syn = _cube(6), _cube(7)
    w2p = O.W2Params(n_xi=300)
    ctx = O.w2_prepare(d, DT, w2p)
    J, w2, _ = O.w2_misfit(ctx, syn, DT, w2p, with_adjoint=False)
    # each W2 against an independent evaluation on the shifted, weighted traces
    for s in range(2):
        for r in range(3):
            ya = ctx.omega[0, s, r] * syn[0, s, r] + ctx.cshift[0, s, r]
            yb = ctx.omega[0, s, r] * d[0, s, r] + ctx.cshift[0, s, r]
            np.testing.assert_allclose(w2[0, s, r], O.w2_signals(ya, yb, DT, nxi=300), rtol=1e-13)
    np.testing.assert_allclose(J[0], w2.sum() / ctx.S_obs[0], rtol=1e-14)


def test_adjoint_source_matches_central_differences():
    d, syn = _cube(8), _cube(9)
    w2p = O.W2Params(n_xi=400)
    ctx = O.w2_prepare(d, DT, w2p)
    J, _, adj = O.w2_misfit(ctx, syn, DT, w2p)
    rng = np.random.default_rng(10)
    for _ in range(3):
        dd = rng.standard_normal(syn.shape)
        h = 1e-7
        Jp = O.w2_misfit(ctx, syn + h * dd, DT, w2p, with_adjoint=False)[0][0]
        Jm = O.w2_misfit(ctx, syn - h * dd, DT, w2p, with_adjoint=False)[0][0]
        fd = (Jp - Jm) / (2 * h)
        an = np.vdot(adj, dd)
        assert abs(fd - an) < 1e-6 * abs(an)
    # single-sample perturbations on one trace, including both ends
    for k in (0, 1, 57, 200, 398, 399):
        e = np.zeros_like(syn)
        e[0, 1, 2, k] = 1.0
        h = 1e-7
        fd = (O.w2_misfit(ctx, syn + h * e, DT, w2p, False)[0][0] -
              O.w2_misfit(ctx, syn - h * e, DT, w2p, False)[0][0]) / (2 * h)
        assert abs(fd - adj[0, 1, 2, k]) < 1e-6 * np.abs(adj[0, 1, 2]).max()


def test_negative_total_mass_density_and_derivative():
    # A synthetic trace can lie mostly below the shift c' taken from the
    # observed data, so that its weighted, shifted values integrate to a
    # negative total Z.  The density map y / (Z + eps') (Eq. pdf_map) still
    # normalises it; with eps' = 0 negating a signal leaves its density, its
    # quantiles and every W2 unchanged.
    ya, yb = gauss(0.40, 0.05), gauss(0.52, 0.03)
    w = O.w2_signals(ya, yb, DT, eps=0.0, nxi=500)
    assert O.w2_signals(-ya, yb, DT, eps=0.0, nxi=500) == w
    assert O.w2_signals(-ya, -yb, DT, eps=0.0, nxi=500) == w
    # translation closed form still holds for the negated pair
    yc = gauss(0.40 + 0.07, 0.05)
    np.testing.assert_allclose(O.w2_signals(-ya, -yc, DT, eps=0.0, nxi=1000), 0.07, rtol=2e-3)
    # the misfit of a cube whose traces have a negative total, and its
    # derivative against central differences
    d = _cube(11)
    syn = -4.0 * np.abs(_cube(12))
    w2p = O.W2Params(n_xi=400)
    ctx = O.w2_prepare(d, DT, w2p)
    y = ctx.omega * syn + ctx.cshift[..., None]
    assert np.all(np.trapezoid(y, dx=DT, axis=-1) < 0)
    J, w2, adj = O.w2_misfit(ctx, syn, DT, w2p)
    assert np.all(np.isfinite(w2)) and J[0] > 0
    rng = np.random.default_rng(13)
    for _ in range(2):
        dd = rng.standard_normal(syn.shape)
        h = 1e-7
        Jp = O.w2_misfit(ctx, syn + h * dd, DT, w2p, with_adjoint=False)[0][0]
        Jm = O.w2_misfit(ctx, syn - h * dd, DT, w2p, with_adjoint=False)[0][0]
        an = np.vdot(adj, dd)
        assert abs((Jp - Jm) / (2 * h) - an) < 1e-6 * abs(an)
