"""GPU parity of the comparison methods' hot-path pieces against the oracle:
the least-squares potential (DPS baseline), the squared unenhanced W2
objective (W2 + TV baseline), the TV subgradient, the reconstruction
measures, and three iterations of the two TV-regularised descent baselines
run through the library against the same loops run by the oracle.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_ADJ, TOL_GRAD, TOL_J, initial, models, problems, rel_l2  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2603_16393_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def H(t):
    return t.double().cpu().numpy()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_l2_misfit_matches_oracle(api):
    gp, op = problems(24, 30, 8, 300, 3, batch=2)
    rng = np.random.default_rng(1)
    d_obs = f32(rng.standard_normal((2, 3, gp.nr, 300)))
    d_syn = f32(d_obs + 0.1 * rng.standard_normal(d_obs.shape))
    with api.Plan(gp) as plan:
        J, adj = plan.l2_misfit(T(d_obs), T(d_syn), sigma=0.05)
        torch.cuda.synchronize()
    J_o, adj_o = O.l2_misfit(d_obs, d_syn, sigma=0.05)
    assert rel_l2(H(J), J_o) <= TOL_J
    assert rel_l2(H(adj), adj_o) <= 1e-6


@pytest.mark.parametrize("ties", [False, True])
def test_tv_grad_matches_oracle(api, ties):
    rng = np.random.default_rng(2)
    if ties:   # integer-valued fields: many equal neighbours (sign(0) = 0)
        v = f32(rng.integers(0, 4, (3, 70, 70)) * 100.0 + 2000.0)
    else:
        v = f32(rng.uniform(1500, 4500, (3, 70, 70)))
    g = f32(rng.standard_normal(v.shape) * 1e-6)
    h, tv = api.tv_grad(T(v), T(g), alpha=0.03, unit=1500.0)
    torch.cuda.synchronize()
    tv_o, h_o = O.tv_grad(v, g, 0.03, 1500.0)
    assert rel_l2(H(tv), tv_o) <= 1e-6
    assert rel_l2(H(h), h_o) <= 1e-6
    h0, _ = api.tv_grad(T(v), None, alpha=0.03, unit=1500.0)
    _, h0_o = O.tv_grad(v, None, 0.03, 1500.0)
    assert rel_l2(H(h0), h0_o) <= 1e-6


def test_image_metrics_match_oracle(api):
    vt = models("curved_faulted", [1, 2, 3], 70, 70)
    vr = f32(vt + I.smooth_perturbation(4, 70, 70, 200.0)[None] +
             np.random.default_rng(5).normal(0, 30, vt.shape))
    for R in (3000.0, 2.0 * 1500.0):
        m = H(api.image_metrics(T(vt), T(vr), R))
        m_o = O.image_metrics(vt, vr, R)
        np.testing.assert_allclose(m[:, :2], m_o[:, :2], rtol=1e-5)
        np.testing.assert_allclose(m[:, 2], m_o[:, 2], atol=1e-5)
    m = H(api.image_metrics(T(vt), T(vt), 3000.0))
    assert np.all(m[:, 0] == 0) and np.all(np.isinf(m[:, 1])) and np.allclose(m[:, 2], 1, atol=1e-6)


def _w2sq(api):
    return api.W2Params(k=0.0, n_xi=400, squared=True), O.W2Params(k=0.0, n_xi=400, squared=True)


def test_squared_w2_misfit_on_shared_data(api):
    gp, op = problems(24, 30, 8, 400, 3, batch=2, f_peak=20.0)
    w2p, ow2 = _w2sq(api)
    d_obs = f32(O.forward(op, models("layered", [5, 6], 24, 30)))
    d_syn = f32(O.forward(op, initial(2, 24, 30)))
    with api.Plan(gp, w2p) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        J, w2, adj = plan.w2_misfit(ctx, T(d_syn))
        J0, _, adj0 = plan.w2_misfit(ctx, T(d_obs))
        torch.cuda.synchronize()
    octx = O.w2_prepare(d_obs, op.dt, ow2)
    J_o, w2_o, adj_o = O.w2_misfit(octx, d_syn, op.dt, ow2)
    assert rel_l2(H(J), J_o) <= TOL_J, (H(J), J_o)
    assert rel_l2(H(w2), w2_o) <= TOL_J
    assert rel_l2(H(adj), adj_o) <= TOL_ADJ
    assert float(J0.abs().max()) == 0 and float(adj0.abs().max()) == 0


def test_squared_w2_gradient_matches_oracle(api):
    nz, nx, nb, nt, ns = 30, 70, 20, 300, 3
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    w2p, ow2 = _w2sq(api)
    d_obs = f32(O.forward(op, models("layered", [7, 8], nz, nx)))
    v0 = initial(2, nz, nx)
    with api.Plan(gp, w2p) as plan:
        J, g, _ = plan.gradient(T(v0), plan.w2_prepare(T(d_obs)))
        torch.cuda.synchronize()
        plan.check()
    J_o, g_o, _ = O.gradient(op, v0, O.w2_prepare(d_obs, op.dt, ow2), ow2)
    assert rel_l2(H(J), J_o) <= TOL_J * 10
    for b in range(2):
        assert rel_l2(H(g)[b], g_o[b]) <= TOL_GRAD, rel_l2(H(g)[b], g_o[b])


def test_l2_potential_gradient_matches_oracle(api):
    from paper_2603_16393_gb300 import baselines
    nz, nx, nb, nt, ns = 24, 30, 8, 300, 3
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=20.0)
    d_obs = f32(O.forward(op, models("curved_faulted", [1, 2], nz, nx)))
    v0 = initial(2, nz, nx)
    with api.Plan(gp) as plan:
        J, g = baselines.l2_gradient(plan, T(v0), T(d_obs), sigma=0.01)
        torch.cuda.synchronize()

    def unit(bs):
        b, s = bs
        d, u_all = O.forward_shot(op, v0[b], s, keep_wavefield=True)
        Jb, adj = O.l2_misfit(d_obs[b, s][None], d[None], sigma=0.01)
        return b, Jb[0], O.fold(op, O.adjoint_shot(op, v0[b], s, adj[0], u_all))
    with ThreadPoolExecutor(O.nthreads()) as ex:
        out = list(ex.map(unit, [(b, s) for b in range(2) for s in range(ns)]))
    J_o = np.array([sum(o[1] for o in out if o[0] == b) for b in range(2)])
    g_o = np.stack([sum(o[2] for o in out if o[0] == b) for b in range(2)])
    assert rel_l2(H(J), J_o) <= TOL_J
    for b in range(2):
        assert rel_l2(H(g)[b], g_o[b]) <= TOL_GRAD


def _oracle_loop(op, ow2, octx, v, alpha, prm, unit, iters):
    for _ in range(iters):
        _, g, _ = O.gradient(op, v, octx, ow2)
        _, h = O.tv_grad(v, g, alpha, unit)
        # the library's update in physical units = the paper's update applied
        # to the normalised field v / unit
        v, _ = O.guided_step(v, v / unit, g * unit, h * unit * unit, O.GuideParams(**prm))
    return v


@pytest.mark.parametrize("which", ["w2_tv", "ot_we_tv"])
def test_descent_baselines_match_the_oracle_loop(api, which):
    from paper_2603_16393_gb300 import baselines
    nz, nx, nb, nt, ns = 24, 30, 8, 300, 3
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=20.0, v_max=4600.0)
    unit, alpha, iters = 1500.0, 0.05, 3
    d_obs = f32(O.forward(op, models("curved_faulted", [3, 4], nz, nx)))
    # start away from ties: the linear initial model has equal neighbours along x
    v0 = f32(initial(2, nz, nx) + np.stack([I.smooth_perturbation(9 + b, nz, nx, 40.0)
                                            for b in range(2)]))
    if which == "w2_tv":
        w2p, ow2 = api.W2Params(k=0.0, squared=True), O.W2Params(k=0.0, squared=True)
        rho0 = 2.0
        prm = dict(rho0=rho0, c=1.0, tau=3.0e38, gamma=0.0)
    else:
        w2p, ow2 = api.W2Params(), O.W2Params()
        prm = dict(rho0=0.5, c=0.1, tau=0.0, gamma=0.55)
    with api.Plan(gp, w2p) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        if which == "w2_tv":
            v, hist = baselines.w2_tv_descent(plan, ctx, T(v0), alpha, rho0, iters, unit=unit)
        else:
            v, hist = baselines.ot_we_tv_descent(plan, ctx, T(v0), alpha,
                                                 api.GuideParams(unit=unit, **prm), iters)
        torch.cuda.synchronize()
        plan.check()
    v_o = _oracle_loop(op, ow2, O.w2_prepare(d_obs, op.dt, ow2), v0, alpha, prm, unit, iters)
    upd, upd_o = H(v) - v0, v_o - v0
    assert np.abs(upd_o).max() > 1.0, np.abs(upd_o).max()     # the loop moved the model
    assert rel_l2(upd, upd_o) <= 1e-3, rel_l2(upd, upd_o)
    J = [float(h[0].sum()) for h in hist]
    assert J[-1] < J[0]
