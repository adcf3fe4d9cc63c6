"""GPU parity of the CPML absorber (fwi_problem.absorber = FWI_ABSORBER_CPML,
its own global-memory kernels) against the FP64 CPML oracle: seismograms,
the adjoint stage on a shared adjoint source, and the whole W2 gradient;
without stretching (refl_R = 1) it is the undamped leapfrog of the sponge
kernels."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_DATA, TOL_GRAD, TOL_J, initial, models, problems, rel_l2  # noqa: E402
from oracle import cpml as C  # noqa: E402
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


def _cpml(api, nz, nx, nb, nt, ns, batch=2, **kw):
    gp, op = problems(nz, nx, nb, nt, ns, batch=batch, f_peak=25.0, **kw)
    return dataclasses.replace(gp, absorber=api.ABSORBER_CPML), op


@pytest.mark.parametrize("nz,nx,nb,nt,ns", [
    (30, 70, 20, 400, 3),
    (41, 37, 12, 300, 2),      # odd sizes, partial 32 x 8 blocks in both directions
])
def test_cpml_forward_matches_oracle(api, nz, nx, nb, nt, ns):
    gp, op = _cpml(api, nz, nx, nb, nt, ns)
    v = models("curved_faulted", [3, 4], nz, nx)
    with api.Plan(gp) as plan:
        assert plan.kernels == api.KERNELS_CPML
        d, _ = plan.forward(T(v))
        torch.cuda.synchronize()
        plan.check()
    d_o = C.forward(op, v)
    assert rel_l2(H(d), d_o) <= TOL_DATA, rel_l2(H(d), d_o)


def test_cpml_without_stretching_is_the_undamped_sponge_path(api):
    nz, nx, nb, nt, ns = 30, 70, 20, 400, 3
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    gp = dataclasses.replace(gp, refl_R=1.0)
    v = T(models("layered", [1, 2], nz, nx))
    out = []
    for absorber in (api.ABSORBER_SPONGE, api.ABSORBER_CPML):
        with api.Plan(dataclasses.replace(gp, absorber=absorber)) as plan:
            out.append(H(plan.forward(v, store=False)[0]))
            torch.cuda.synchronize()
            plan.check()
    assert rel_l2(out[1], out[0]) <= TOL_DATA


def test_cpml_adjoint_stage_matches_oracle(api):
    nz, nx, nb, nt, ns = 30, 70, 20, 300, 2
    gp, op = _cpml(api, nz, nx, nb, nt, ns)
    v0 = initial(2, nz, nx)
    adj = np.random.default_rng(5).standard_normal((2, ns, gp.nr, nt))
    adj = adj.astype(np.float32).astype(np.float64)
    with api.Plan(gp) as plan:
        plan.forward(T(v0))
        g = H(plan.adjoint_grad(T(v0), T(adj)))
        torch.cuda.synchronize()
        plan.check()
    for b in range(2):
        g_o = np.zeros((nz, nx))
        for s in range(ns):
            _, rec = C.forward_shot(op, v0[b], s, keep_record=True)
            g_o += O.fold(op, C.adjoint_shot(op, v0[b], s, adj[b, s], rec))
        assert rel_l2(g[b], g_o) <= TOL_GRAD, (b, rel_l2(g[b], g_o))


def test_cpml_gradient_matches_oracle(api):
    nz, nx, nb, nt, ns = 30, 70, 20, 400, 3
    gp, op = _cpml(api, nz, nx, nb, nt, ns)
    w2p, ow2 = api.W2Params(n_xi=400), O.W2Params(n_xi=400)
    vt = models("layered", [7, 8], nz, nx)
    v0 = initial(2, nz, nx)
    d_obs = C.forward(op, vt).astype(np.float32).astype(np.float64)
    with api.Plan(gp, w2p) as plan:
        J, g, _ = plan.gradient(T(v0), plan.w2_prepare(T(d_obs)))
        torch.cuda.synchronize()
        plan.check()
    J_o, g_o = C.gradient(op, v0, O.w2_prepare(d_obs, op.dt, ow2), ow2)
    assert rel_l2(H(J), J_o) <= TOL_J * 10, (H(J), J_o)
    for b in range(2):
        assert rel_l2(H(g)[b], g_o[b]) <= TOL_GRAD, (b, rel_l2(H(g)[b], g_o[b]))
