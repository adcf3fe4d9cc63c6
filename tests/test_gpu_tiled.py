"""GPU parity of the propagators for padded grids beyond one CTA's shared
memory against the FP64 oracle: the global-memory tiled kernels and the
cluster kernels (rows split over 8 CTAs, halos through distributed shared
memory), each forced through fwi_problem.kernels.

100 x 140 models with a 20-cell layer pad to 120 x 180 cells: 4 x 3 tiles of
32 x 64 with ragged last tiles in both directions, a cluster of 5 CTAs of 26
rows (the last holds 16) in single-column strips or of 6 CTAs of 20 rows in
column pairs, and too large for the shared-memory resident kernels (two
levels + a table = 269 KB).  The cluster kernels run in both thread shapes:
column pairs (the default for an even padded width; the odd one of 321 falls
back to single columns) and single-column strips.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_DATA, TOL_GRAD, TOL_J, initial, models, problems, rel_l2  # noqa: E402
from oracle import oracle as O  # noqa: E402

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


FAMILIES = ("tiled", "tiled_quads", "cluster", "cluster_columns")


def _fam(api, name):
    return {"tiled": api.KERNELS_TILED, "tiled_quads": api.KERNELS_TILED,
            "cluster": api.KERNELS_CLUSTER, "cluster_columns": api.KERNELS_CLUSTER}[name]


def _forced(api, gp, fam):
    """gp on the family `fam`: "cluster" takes the default shape (column pairs
    where the padded width is even), "cluster_columns" the single-column
    strips (13 rows where they fit, else 19), "tiled" the scalar 8-row threads
    and "tiled_quads" the float4 column quads (the default) of the tiled
    kernels."""
    gp = dataclasses.replace(gp, kernels=_fam(api, fam))
    if fam == "tiled_quads":
        return dataclasses.replace(gp, shape=api.SHAPE_TILED_QUADS)
    if fam == "tiled":
        return dataclasses.replace(gp, shape=api.SHAPE_TILED_ROWS8)
    if fam != "cluster_columns":
        return gp
    try:
        api.fwi_plan_create(dataclasses.replace(gp, shape=api.SHAPE_CLUSTER_RS13),
                            api.W2Params())
        return dataclasses.replace(gp, shape=api.SHAPE_CLUSTER_RS13)
    except api.FwiError:
        return dataclasses.replace(gp, shape=api.SHAPE_CLUSTER_RS19)


@pytest.mark.parametrize("fam", FAMILIES)
@pytest.mark.parametrize("nz,nx,nb,nt,ns,top_bc", [
    (100, 140, 20, 500, 3, 0),
    (100, 140, 20, 500, 2, 1),
    (90, 301, 10, 300, 2, 0),      # odd padded width (321; tiled row pitch 324); 8 CTAs of 13 rows
    (250, 60, 12, 300, 2, 1),      # 262 x 84 cells: 7 CTAs of three 13-row strips, the last 28 rows
    (230, 270, 15, 300, 2, 1),     # 245 x 300 cells: 7 CTAs of two 19-row strips, the last 17 rows
])
def test_tiled_forward_matches_oracle(api, nz, nx, nb, nt, ns, top_bc, fam):
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc)
    gp = _forced(api, gp, fam)
    v = models("curved_faulted", [3, 4], nz, nx)
    with api.Plan(gp) as plan:
        assert plan.kernels == _fam(api, fam)
        d, _ = plan.forward(T(v))
        torch.cuda.synchronize()
        plan.check()
    d_o = O.forward(op, v)
    err = rel_l2(H(d), d_o)
    assert err <= TOL_DATA, err


@pytest.mark.parametrize("fam", FAMILIES)
@pytest.mark.parametrize("top_bc", [0, 1])
def test_tiled_gradient_matches_oracle(api, top_bc, fam):
    nz, nx, nb, nt, ns = 100, 140, 20, 500, 3
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc)
    gp = _forced(api, gp, fam)
    w2p, ow2 = api.W2Params(n_xi=500), O.W2Params(n_xi=500)
    vt = models("layered", [7, 8], nz, nx)
    v0 = initial(2, nz, nx)
    d_obs = O.forward(op, vt).astype(np.float32).astype(np.float64)
    with api.Plan(gp, w2p) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        J, g, _ = plan.gradient(T(v0), ctx)
        torch.cuda.synchronize()
        plan.check()
    octx = O.w2_prepare(d_obs, op.dt, ow2)
    J_o, g_o, _ = O.gradient(op, v0, octx, ow2)
    assert rel_l2(H(J), J_o) <= TOL_J * 10, (H(J), J_o)
    for b in range(2):
        assert rel_l2(H(g)[b], g_o[b]) <= TOL_GRAD, (b, rel_l2(H(g)[b], g_o[b]))


def test_tiled_checkpoints_are_bitwise_store_all(api):
    nz, nx, nb, nt, ns = 100, 140, 20, 300, 2
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    w2p = api.W2Params(n_xi=400)
    vt = models("layered", [1, 2], nz, nx)
    v0 = initial(2, nz, nx)
    gp = dataclasses.replace(gp, kernels=api.KERNELS_TILED)
    out = []
    for K in (0, 37):
        with api.Plan(dataclasses.replace(gp, checkpoint_every=K), w2p) as plan:
            d_obs, _ = plan.forward(T(vt), store=False)
            ctx = plan.w2_prepare(d_obs.clone())
            J, g, _ = plan.gradient(T(v0), ctx)
            torch.cuda.synchronize()
            plan.check()
            out.append((J, g))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_tiled_autograd_is_the_library_gradient(api):
    from paper_2603_16393_gb300 import autograd as G
    nz, nx, nb, nt, ns = 100, 140, 20, 300, 2
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    gp = dataclasses.replace(gp, checkpoint_every=64)
    with api.Plan(gp, api.W2Params(n_xi=400), snapshots=False) as plan:
        d_obs, _ = plan.forward(T(models("layered", [1, 2], nz, nx)), store=False)
        ctx = plan.w2_prepare(d_obs.clone())
        v = T(initial(2, nz, nx)).requires_grad_(True)
        J = G.w2_fwi_objective(v, plan, ctx)
        J.sum().backward()
        plan2 = api.Plan(gp, api.W2Params(n_xi=400))
        J2, g2, _ = plan2.gradient(v.detach(), ctx)
        torch.cuda.synchronize()
    assert torch.equal(J.detach(), J2) and torch.equal(v.grad, g2)


# ---------------------------------------------------------------- 8th-order stencil

def _order8(gp, op):
    return dataclasses.replace(gp, space_order=8), dataclasses.replace(op, space_order=8)


@pytest.mark.parametrize("nz,nx,nb,nt,ns,top_bc", [
    (30, 70, 20, 300, 3, 0),      # a grid the 4th-order path keeps in shared memory
    (41, 64, 25, 260, 2, 1),      # mirrored top over four rows
    (100, 140, 20, 400, 2, 0),
])
def test_order8_forward_matches_oracle(api, nz, nx, nb, nt, ns, top_bc):
    gp, op = _order8(*problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc))
    v = models("curved_faulted", [3, 4], nz, nx)
    with api.Plan(gp) as plan:
        d, _ = plan.forward(T(v))
        torch.cuda.synchronize()
        plan.check()
    d_o = O.forward(op, v)
    assert rel_l2(H(d), d_o) <= TOL_DATA, rel_l2(H(d), d_o)
    # and it is not the 4th-order result
    assert rel_l2(d_o, O.forward(dataclasses.replace(op, space_order=4), v)) > 1e-3


@pytest.mark.parametrize("top_bc", [0, 1])
def test_order8_gradient_matches_oracle(api, top_bc):
    nz, nx, nb, nt, ns = 30, 70, 20, 300, 3
    gp, op = _order8(*problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc))
    w2p, ow2 = api.W2Params(n_xi=400), O.W2Params(n_xi=400)
    vt = models("layered", [7, 8], nz, nx)
    v0 = initial(2, nz, nx)
    d_obs = O.forward(op, vt).astype(np.float32).astype(np.float64)
    out = []
    for K in (0, 41):
        with api.Plan(dataclasses.replace(gp, checkpoint_every=K), w2p) as plan:
            J, g, _ = plan.gradient(T(v0), plan.w2_prepare(T(d_obs)))
            torch.cuda.synchronize()
            plan.check()
            out.append((J, g))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    J, g = H(out[0][0]), H(out[0][1])
    J_o, g_o, _ = O.gradient(op, v0, O.w2_prepare(d_obs, op.dt, ow2), ow2)
    assert rel_l2(J, J_o) <= TOL_J * 10, (J, J_o)
    for b in range(2):
        assert rel_l2(g[b], g_o[b]) <= TOL_GRAD, (b, rel_l2(g[b], g_o[b]))


@pytest.mark.parametrize("top_bc", [0, 1])
def test_cluster_gradient_agrees_with_the_tiled_gradient(api, top_bc):
    # the same recurrences on two kernel families: float rounding apart
    # (136 x 232 cells: 6 CTAs of 26 rows, the last holding 6)
    nz, nx, nb, nt, ns = 120, 200, 16, 400, 3
    gp, _ = problems(nz, nx, nb, nt, ns, batch=3, f_peak=25.0, top_bc=top_bc)
    w2p = api.W2Params(n_xi=400)
    vt = models("curved_faulted", [1, 2, 3], nz, nx)
    v0 = initial(3, nz, nx)
    res = {}
    for fam in FAMILIES:
        with api.Plan(_forced(api, gp, fam), w2p) as plan:
            d_obs, _ = plan.forward(T(vt), store=False)
            ctx = plan.w2_prepare(d_obs.clone())
            J, g, _ = plan.gradient(T(v0), ctx)
            torch.cuda.synchronize()
            plan.check()
            res[fam] = (H(d_obs), H(J), H(g))
    for c in ("cluster", "cluster_columns"):
        assert rel_l2(res[c][0], res["tiled"][0]) <= 1e-5
        assert rel_l2(res[c][1], res["tiled"][1]) <= 1e-4
        for b in range(3):
            assert rel_l2(res[c][2][b], res["tiled"][2][b]) <= 1e-3
    # column pairs and single columns: per cell the same operations in the same
    # order, so the same bits (the reflecting top); the mirrored top's
    # transposed correction leaves its two products to the compiler's
    # contraction in the single-column adjoint, a rounding difference at rows
    # 1 and 2 every step (1.7e-5 measured after 400 steps): the gradient bar
    # the tiled kernels' column quads: the same operations per cell, the same bits
    for k in range(3):
        assert np.array_equal(res["tiled_quads"][k], res["tiled"][k])
    assert np.array_equal(res["cluster"][0], res["cluster_columns"][0])
    if top_bc == 0:
        assert np.array_equal(res["cluster"][1], res["cluster_columns"][1])
        assert np.array_equal(res["cluster"][2], res["cluster_columns"][2])
    else:
        assert rel_l2(res["cluster"][2], res["cluster_columns"][2]) <= TOL_GRAD


@pytest.mark.parametrize("top_bc", [0, 1])
@pytest.mark.parametrize("order", [4, 8])
def test_tiled_quads_are_bitwise_the_scalar_tiled_kernels(api, order, top_bc):
    # data, J and dJ/dv of the float4 column quads against the 8-row scalar
    # threads, with checkpoints (K = 13) so that resume and recompute run too
    nz, nx, nb, nt, ns = 45, 77, 9, 200, 2       # 54 x 95 cells: ragged tiles, pad columns
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc)
    gp = dataclasses.replace(gp, kernels=api.KERNELS_TILED, space_order=order, checkpoint_every=13)
    vt = T(models("curved_faulted", [5, 6], nz, nx))
    v0 = T(initial(2, nz, nx))
    out = []
    for sh in (api.SHAPE_TILED_ROWS8, api.SHAPE_TILED_QUADS):
        with api.Plan(dataclasses.replace(gp, shape=sh), api.W2Params(n_xi=300)) as plan:
            d_obs, _ = plan.forward(vt, store=False)
            J, g, _ = plan.gradient(v0, plan.w2_prepare(d_obs.clone()))
            torch.cuda.synchronize()
            plan.check()
            out.append((H(d_obs), H(J), H(g)))
    for k in range(3):
        assert np.array_equal(out[0][k], out[1][k]), k
