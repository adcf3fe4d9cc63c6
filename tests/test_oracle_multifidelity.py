"""Pins of the low-fidelity surrogate's oracle (``oracle/multifidelity.py``),
CPU only: the restriction against brute-force block means, its transpose
against the explicit matrix's transpose, constants and the dot-product
identity, the decimation's time alignment against a coarse run of the same
physics, and central differences of the composite surrogate potential."""
import numpy as np
import pytest

from oracle import multifidelity as M
from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I


@pytest.mark.parametrize("nz,nx", [(4, 6), (5, 7), (1, 3), (70, 70)])
def test_restriction_is_the_block_mean(nz, nx):
    rng = np.random.default_rng(nz * nx)
    v = rng.standard_normal((2, nz, nx))
    r = M.restrict(v)
    nzc, nxc = M.coarse_shape(nz, nx)
    assert r.shape == (2, nzc, nxc)
    for I_ in range(nzc):
        for J in range(nxc):
            cells = [v[:, i, j] for i in (2 * I_, 2 * I_ + 1) for j in (2 * J, 2 * J + 1)
                     if i < nz and j < nx]
            np.testing.assert_allclose(r[:, I_, J], np.mean(cells, axis=0), rtol=0, atol=1e-14)
    np.testing.assert_allclose(M.restrict(np.full((1, nz, nx), 3.25)), 3.25, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nz,nx", [(4, 6), (5, 7), (3, 1)])
def test_transpose_is_the_matrix_transpose(nz, nx):
    nzc, nxc = M.coarse_shape(nz, nx)
    R = np.zeros((nzc * nxc, nz * nx))
    for k in range(nz * nx):
        e = np.zeros(nz * nx)
        e[k] = 1.0
        R[:, k] = M.restrict(e.reshape(1, nz, nx)).ravel()
    RT = np.zeros((nz * nx, nzc * nxc))
    for k in range(nzc * nxc):
        e = np.zeros(nzc * nxc)
        e[k] = 1.0
        RT[:, k] = M.restrict_transpose(e.reshape(1, nzc, nxc), nz, nx).ravel()
    np.testing.assert_allclose(RT, R.T, rtol=0, atol=1e-15)


def test_decimation_matches_a_coarse_run_of_the_same_physics():
    # a homogeneous medium with the mirrored top (its boundary lies on row 0
    # at every resolution) and receivers below the surface: the coarse run's
    # sample m is closest to the fine run's sample 2m + 1 (same time), the gap
    # shrinks as both grids are refined, and the other alignment (2m) is
    # farther at every resolution
    def gaps(nz, nt, dx, dt):
        fine = O.Problem(nz=nz, nx=nz, nb=8, nt=nt, dz=dx, dx=dx, dt=dt, src_iz=[nz // 2],
                         src_ix=[nz // 2], rec_iz=[nz // 5] * nz, rec_ix=list(range(nz)),
                         f_peak=15.0, top_bc=1)
        coarse = M.coarse_problem(fine)
        v = np.full((1, nz, nz), 2000.0)
        df = O.forward(fine, v, threads=1)
        dc = O.forward(coarse, M.restrict(v), threads=1)
        dd = M.decimate(df)
        other = df[:, :, ::2, 0:2 * (nt // 2):2]
        assert dd.shape == dc.shape == other.shape
        rel = lambda a: np.linalg.norm(a - dc) / np.linalg.norm(a)  # noqa: E731
        return rel(dd), rel(other)
    e1, o1 = gaps(20, 240, 10.0, 1e-3)
    e2, o2 = gaps(40, 480, 5.0, 5e-4)
    assert e1 < o1 and e2 < o2, (e1, o1, e2, o2)
    assert e2 < 0.8 * e1 and e1 < 0.25, (e1, e2)


def test_decimation_keeps_even_receivers_and_odd_samples():
    d = np.arange(2 * 1 * 5 * 7, dtype=float).reshape(2, 1, 5, 7)
    dc = M.decimate(d)
    assert dc.shape == (2, 1, 3, 3)
    np.testing.assert_array_equal(dc[1, 0, 2], d[1, 0, 4, [1, 3, 5]])


def test_surrogate_gradient_matches_central_differences():
    g = I.surface_geometry(12, 1)
    prob = O.Problem(nz=12, nx=12, nb=4, nt=120, dz=10.0, dx=10.0, dt=1e-3,
                     src_iz=g.src_iz, src_ix=g.src_ix, rec_iz=g.rec_iz, rec_ix=g.rec_ix,
                     f_peak=30.0, v_ref=2500.0)
    w2p = O.W2Params(n_xi=200)
    vt = 1800 + 400 * I.layered_model(1, 12, 12) / 4500.0 + I.smooth_perturbation(5, 12, 12, 150)
    pot = M.surrogate_potential(prob, O.forward(prob, vt[None]), w2p, threads=1)
    v = 2000 + I.smooth_perturbation(6, 12, 12, 100)
    J, grad = pot(v[None])
    assert J[0] > 0
    h = 1e-3
    fd = np.zeros_like(v)
    for iz in range(12):
        for ix in range(12):
            e = np.zeros_like(v)
            e[iz, ix] = h
            fd[iz, ix] = (pot((v + e)[None])[0][0] - pot((v - e)[None])[0][0]) / (2 * h)
    rel = np.linalg.norm(fd - grad[0]) / np.linalg.norm(fd)
    assert rel < 1e-6, rel
