"""GPU parity at the edges of the input space, against the FP64 oracle:
the shortest time axis with a single shot and receiver, no absorbing layer,
traces that are exactly zero in both observed and synthetic data (the W2
density then has Z = 0: every quantile clamps to the last sample), and the
largest acquisitions the ABI accepts (FWI_MAX_SHOTS shots, FWI_MAX_RECEIVERS
receivers on the tiled kernels)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import (TOL_ADJ, TOL_DATA, TOL_GRAD, TOL_GRAD_W2, TOL_J, initial, models,  # noqa: E402
                       problems, rel_l2)
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


def _gradient_pair(api, gp, op, vt, v0, nxi=200):
    w2p, ow2 = api.W2Params(n_xi=nxi), O.W2Params(n_xi=nxi)
    d_obs = O.forward(op, vt).astype(np.float32).astype(np.float64)
    B = vt.shape[0]
    with api.Plan(gp, w2p) as plan:
        J, g, w2 = plan.gradient(T(v0), plan.w2_prepare(T(d_obs)))
        torch.cuda.synchronize()
        plan.check()
    J_o, g_o, w2_o = O.gradient(op, v0, O.w2_prepare(d_obs, op.dt, ow2), ow2)
    return H(J), H(g), H(w2), J_o, g_o, w2_o, B


@pytest.mark.parametrize("nt", [2, 3])
def test_shortest_time_axis_one_shot_one_receiver(api, nt):
    # two samples: the receiver 1 cell from the source sees the wave at once
    geo = I.Geometry(src_iz=(3,), src_ix=(5,), rec_iz=(3,), rec_ix=(6,))
    gp, op = problems(9, 11, 4, nt, 1, batch=2, f_peak=25.0, geo=geo)
    gp = dataclasses.replace(gp, t0=0.001)
    op = dataclasses.replace(op, t0=0.001)
    vt, v0 = models("layered", [1, 2], 9, 11), initial(2, 9, 11)
    with api.Plan(gp) as plan:
        d = H(plan.forward(T(vt))[0])
        torch.cuda.synchronize()
        plan.check()
    d_o = O.forward(op, vt)
    assert np.abs(d_o).max() > 0
    assert rel_l2(d, d_o) <= TOL_DATA
    J, g, w2, J_o, g_o, w2_o, B = _gradient_pair(api, gp, op, vt, v0, nxi=64)
    assert rel_l2(J, J_o) <= TOL_J * 10, (J, J_o)
    for b in range(B):
        if np.abs(g_o[b]).max() > 0:
            assert rel_l2(g[b], g_o[b]) <= TOL_GRAD * 10, (b, rel_l2(g[b], g_o[b]))


def test_no_absorbing_layer(api):
    # a fully reflecting box: every stage at its own bar; end to end, the
    # GPU's 4e-7 data difference moves one instance's W2 adjoint source by
    # 2e-3 (interpolated quantiles of a reverberant trace change bracket), the
    # conditioning bound of the larger workloads
    gp, op = problems(24, 30, 0, 300, 3, batch=2, f_peak=25.0)
    vt, v0 = models("layered", [3, 4], 24, 30), initial(2, 24, 30)
    w2p, ow2 = api.W2Params(n_xi=200), O.W2Params(n_xi=200)
    d_obs = O.forward(op, vt).astype(np.float32).astype(np.float64)
    d_syn = O.forward(op, v0)
    d_syn32 = d_syn.astype(np.float32).astype(np.float64)
    octx = O.w2_prepare(d_obs, op.dt, ow2)
    _, _, adj_o = O.w2_misfit(octx, d_syn32, op.dt, ow2)
    rnd = np.random.default_rng(0).standard_normal(adj_o.shape).astype(np.float32).astype(np.float64)
    with api.Plan(gp, w2p) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        d = H(plan.forward(T(v0))[0])
        _, _, adj = plan.w2_misfit(ctx, T(d_syn32))
        g_rnd = H(plan.adjoint_grad(T(v0), T(rnd)))
        g_w2 = H(plan.adjoint_grad(T(v0), T(adj_o)))
        J, g, _ = plan.gradient(T(v0), ctx)
        torch.cuda.synchronize()
        plan.check()
    assert rel_l2(d, d_syn) <= TOL_DATA
    assert rel_l2(H(adj), adj_o) <= TOL_ADJ
    for src, g_gpu in ((rnd, g_rnd), (adj_o, g_w2)):
        for b in range(2):
            g_or = sum(O.fold(op, O.adjoint_shot(op, v0[b], s, src[b, s],
                                                 O.forward_shot(op, v0[b], s, True)[1]))
                       for s in range(3))
            assert rel_l2(g_gpu[b], g_or) <= TOL_GRAD, (b, rel_l2(g_gpu[b], g_or))
    J_o, g_o, _ = O.gradient(op, v0, octx, ow2)
    assert rel_l2(H(J), J_o) <= TOL_J * 10
    for b in range(2):
        assert rel_l2(H(g)[b], g_o[b]) <= TOL_GRAD_W2, (b, rel_l2(H(g)[b], g_o[b]))


def test_traces_that_are_exactly_zero(api):
    # 30 steps move a 4th-order stencil's support 60 cells: receivers 61..69
    # of a source at column 0 record exact zeros in both data cubes
    geo = I.Geometry(src_iz=(0,), src_ix=(0,), rec_iz=(0,) * 70, rec_ix=tuple(range(70)))
    gp, op = problems(20, 70, 10, 30, 1, batch=2, f_peak=40.0, geo=geo)
    vt, v0 = models("layered", [5, 6], 20, 70), initial(2, 20, 70)
    d_obs = O.forward(op, vt).astype(np.float32).astype(np.float64)
    d_syn = O.forward(op, v0).astype(np.float32).astype(np.float64)
    assert np.all(d_obs[:, 0, 61:] == 0) and np.all(d_syn[:, 0, 61:] == 0)
    w2p, ow2 = api.W2Params(n_xi=300), O.W2Params(n_xi=300)
    with api.Plan(gp, w2p) as plan:
        J, w2, adj = plan.w2_misfit(plan.w2_prepare(T(d_obs)), T(d_syn))
        torch.cuda.synchronize()
    J_o, w2_o, adj_o = O.w2_misfit(O.w2_prepare(d_obs, op.dt, ow2), d_syn, op.dt, ow2)
    assert np.all(H(w2)[:, 0, 61:] == 0) and np.all(H(adj)[:, 0, 61:] == 0)
    assert rel_l2(H(J), J_o) <= TOL_J
    assert rel_l2(H(w2), w2_o) <= TOL_J
    assert rel_l2(H(adj), adj_o) <= TOL_ADJ


def test_most_shots(api):
    ns = 256                                   # FWI_MAX_SHOTS
    geo = I.Geometry(src_iz=tuple(i % 5 for i in range(ns)), src_ix=tuple(i % 16 for i in range(ns)),
                     rec_iz=(0,) * 16, rec_ix=tuple(range(16)))
    gp, op = problems(8, 16, 4, 120, ns, batch=1, f_peak=30.0, geo=geo)
    v = models("layered", [2], 8, 16)
    with api.Plan(gp) as plan:
        d = H(plan.forward(T(v))[0])
        torch.cuda.synchronize()
        plan.check()
    assert rel_l2(d, O.forward(op, v)) <= TOL_DATA


def test_most_receivers_on_the_tiled_kernels(api):
    nr = 1024                                  # FWI_MAX_RECEIVERS
    geo = I.surface_geometry(1024, 2, nr)
    gp, op = problems(6, 1024, 4, 80, 2, batch=1, f_peak=30.0, geo=geo)
    gp = dataclasses.replace(gp, kernels=api.KERNELS_TILED)
    v = models("layered", [9], 6, 1024)
    with api.Plan(gp) as plan:
        d = H(plan.forward(T(v))[0])
        torch.cuda.synchronize()
        plan.check()
    d_o = O.forward(op, v)
    assert rel_l2(d, d_o) <= TOL_DATA
    w2p, ow2 = api.W2Params(n_xi=100), O.W2Params(n_xi=100)
    d_obs = d_o.astype(np.float32).astype(np.float64)
    d_syn = O.forward(op, v * 1.02).astype(np.float32).astype(np.float64)
    with api.Plan(gp, w2p) as plan:
        J, w2, adj = plan.w2_misfit(plan.w2_prepare(T(d_obs)), T(d_syn))
        torch.cuda.synchronize()
    J_o, w2_o, adj_o = O.w2_misfit(O.w2_prepare(d_obs, op.dt, ow2), d_syn, op.dt, ow2)
    assert rel_l2(H(J), J_o) <= TOL_J
    assert rel_l2(H(adj), adj_o) <= TOL_ADJ
