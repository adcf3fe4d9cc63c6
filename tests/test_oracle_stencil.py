"""Pins of the oracle's spatial operators (CPU only).

P-1: the 4th-order Laplacian is exact on polynomials of degree <= 5 and has
the known error -8 h^4 on x^6 (Taylor expansion of the weights
(-1/12, 4/3, -5/2, 4/3, -1/12)).  The padding and the fold are checked
against numpy's edge padding and its exact transpose.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _grid(NZ, NX, h):
    z = np.arange(NZ)[:, None] * h + 0.0 * np.arange(NX)[None, :]
    x = np.arange(NX)[None, :] * h + 0.0 * np.arange(NZ)[:, None]
    return z, x


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5])
def test_laplacian_exact_on_polynomials_x(k):
    NZ, NX, h = 9, 16, 0.5
    z, x = _grid(NZ, NX, h)
    u = (x + 1.0) ** k
    lap = O.laplacian(u, dz=h, dx=h)
    exact = k * (k - 1) * (x + 1.0) ** (k - 2) if k >= 2 else 0 * x
    # interior: two cells away from every edge (the zero ghosts only act there)
    np.testing.assert_allclose(lap[2:-2, 2:-2], exact[2:-2, 2:-2], rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_laplacian_exact_on_polynomials_z(k):
    NZ, NX, h = 14, 9, 0.25
    z, x = _grid(NZ, NX, h)
    u = (z + 0.5) ** k
    lap = O.laplacian(u, dz=h, dx=2 * h)
    exact = k * (k - 1) * (z + 0.5) ** (k - 2)
    np.testing.assert_allclose(lap[2:-2, 2:-2], exact[2:-2, 2:-2], rtol=1e-11, atol=1e-9)


def test_laplacian_sixth_degree_error():
    # sum_m w_m m^6 = -8, so L x^6 = 30 x^4 - 8 h^4 exactly
    NZ, NX, h = 7, 12, 1.0
    z, x = _grid(NZ, NX, h)
    lap = O.laplacian(x ** 6, dz=h, dx=h)
    np.testing.assert_allclose(lap[2:-2, 2:-2], (30 * x ** 4 - 8 * h ** 4)[2:-2, 2:-2], rtol=1e-13)


def test_laplacian_mixed_and_anisotropic():
    NZ, NX, dz, dx = 12, 13, 0.3, 0.7
    z, x = _grid(NZ, NX, 1.0)
    z, x = z * dz, x * dx
    u = x ** 3 * z ** 2 + 2 * x * z
    exact = 6 * x * z ** 2 + 2 * x ** 3
    lap = O.laplacian(u, dz=dz, dx=dx)
    np.testing.assert_allclose(lap[2:-2, 2:-2], exact[2:-2, 2:-2], rtol=1e-10, atol=1e-9)


def test_zero_ghosts_on_all_sides():
    # a single unit spike next to the corner: L touches only cells within 2
    NZ, NX = 6, 7
    u = np.zeros((NZ, NX))
    u[0, 0] = 1.0
    lap = O.laplacian(u, dz=1.0, dx=1.0)
    expect = np.zeros((NZ, NX))
    expect[0, 0] = -5.0
    expect[0, 1] = expect[1, 0] = 4.0 / 3.0
    expect[0, 2] = expect[2, 0] = -1.0 / 12.0
    np.testing.assert_allclose(lap, expect, atol=1e-15)


def test_mirror_top_is_exact_for_even_functions():
    # top_bc = 1 mirrors rows 1, 2 into the ghosts (du/dn = 0, Eq. 1); an even
    # function of z is then differentiated exactly at rows 0 and 1 as well
    NZ, NX, h = 12, 8, 1.0
    z, x = _grid(NZ, NX, h)
    for u, exact in ((z ** 2, 2 + 0 * z), (z ** 4, 12 * z ** 2)):
        lap = O.laplacian(u, dz=h, dx=h, top_bc=1)
        np.testing.assert_allclose(lap[0:4, 2:-2], exact[0:4, 2:-2], rtol=1e-12, atol=1e-11)
        lap0 = O.laplacian(u, dz=h, dx=h, top_bc=0)
        assert not np.allclose(lap0[0:2, 2:-2], exact[0:2, 2:-2])


@pytest.mark.parametrize("top_bc", [0, 1])
def test_transpose_identity(top_bc):
    rng = np.random.default_rng(1)
    u = rng.standard_normal((11, 9))
    w = rng.standard_normal((11, 9))
    Lu = O.laplacian(u, 0.7, 1.3, top_bc)
    LTw = O.laplacian(w, 0.7, 1.3, top_bc, transpose=True)
    assert abs(np.vdot(Lu, w) - np.vdot(u, LTw)) < 1e-12 * np.abs(Lu).sum() * np.abs(w).max()
    if top_bc == 0:
        np.testing.assert_allclose(LTw, O.laplacian(w, 0.7, 1.3, 0), rtol=1e-14, atol=1e-13)


def test_pad_matches_edge_padding_and_fold_is_its_transpose():
    prob = O.Problem(nz=7, nx=5, nb=3, nt=1, dz=1, dx=1, dt=1, src_iz=(0,), src_ix=(0,),
                     rec_iz=(0,), rec_ix=(0,))
    rng = np.random.default_rng(2)
    v = rng.standard_normal((7, 5))
    vpad = O.pad_model(prob, v)
    np.testing.assert_array_equal(vpad, np.pad(v, ((0, 3), (3, 3)), mode="edge"))
    w = rng.standard_normal(vpad.shape)
    assert abs(np.vdot(vpad, w) - np.vdot(v, O.fold(prob, w))) < 1e-12


def test_damping_profile_shape():
    # zero inside the physical grid, growing quadratically into the layer,
    # no layer above row 0 (reflecting top of Eq. 1)
    prob = O.Problem(nz=6, nx=5, nb=4, nt=1, dz=10, dx=10, dt=1e-3, src_iz=(0,), src_ix=(0,),
                     rec_iz=(0,), rec_ix=(0,), v_ref=3000.0, refl_R=1e-3)
    eta = O.damping(prob)
    assert np.all(eta[:6, 4:9] == 0)
    assert np.all(eta[0:6, 0] > eta[0:6, 1]) and np.all(eta[0:6, 1] > 0)
    e0 = eta[0, 0]
    np.testing.assert_allclose(eta[0, 1:4], e0 * (np.array([3, 2, 1]) / 4.0) ** 2, rtol=1e-14)
    np.testing.assert_allclose(eta[6:, 6], e0 * (np.arange(1, 5) / 4.0) ** 2, rtol=1e-14)
    np.testing.assert_allclose(eta[-1, 0], 2 * e0, rtol=1e-14)
    # the damped wave u_tt + eta u_t = ... loses amplitude as exp(-int eta/2 dt);
    # over a two-way trip through the layer at speed v_ref that factor is R
    L = prob.nb * prob.dx
    two_way = 2 * np.trapezoid(e0 * (np.linspace(0, 1, 2001)) ** 2, dx=L / 2000) / prob.v_ref
    np.testing.assert_allclose(np.exp(-two_way / 2), prob.refl_R, rtol=1e-6)
