"""fwi_w2_misfit_static, the misfit entry point for callers that cannot hand
device memory to the library (a host framework that owns every allocation
through its own pool, a steady-state loop where nothing may be allocated): its
per-trace scratch is an array compiled into the library instead of the
caller's workspace.

Checked through the C ABI against fwi_w2_misfit on the same inputs, on two
calls in a row (the shared array keeps the previous call's contents, so the
second call shows that nothing stale leaks in), and its size limit.  This file
is collected last so that a failure here stops a -x run only after every other
test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_ADJ, TOL_J, models, problems  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_scratch_misfit_matches_workspace_misfit(api):
    dev = torch.device("cuda:0")
    nz, nx, nb, nt, ns = 24, 30, 8, 400, 3
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=20.0)
    vt = models("layered", [5, 6], nz, nx)
    T = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    with api.Plan(gp, api.W2Params(n_xi=500)) as plan:
        d_obs, _ = plan.forward(T(vt), store=False)
        d_obs = d_obs.clone()
        ctx = plan.w2_prepare(d_obs)
        for seeds in ([7, 8], [9, 10]):        # two calls in a row, different data
            v = models("curved_faulted", seeds, nz, nx)
            d_syn, _ = plan.forward(T(v), store=False)
            J_ref, w2_ref, adj_ref = plan.w2_misfit(ctx, d_syn)
            J = torch.empty_like(J_ref)
            w2 = torch.empty_like(w2_ref)
            adj = torch.empty_like(adj_ref)
            api.fwi_w2_misfit_static(plan.handle, ctx, d_syn, J, w2, adj)
            # without per-trace output the scratch alone carries W2 to J; the
            # call reserves no device memory (the driver's free-memory count
            # and torch's allocator are unchanged across it)
            J2 = torch.full_like(J_ref, float("nan"))
            torch.cuda.synchronize()
            free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            api.fwi_w2_misfit_static(plan.handle, ctx, d_syn, J2, None, None)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
            assert _rel(J, J_ref) <= TOL_J and _rel(J2, J_ref) <= TOL_J
            assert _rel(w2, w2_ref) <= TOL_J
            assert _rel(adj, adj_ref) <= TOL_ADJ
            assert torch.isfinite(J2).all()


def test_static_scratch_rejects_too_many_traces(api):
    # batch x ns x nr above the built-in scratch: a clear error, nothing launched
    nx, ns = 70, 5
    batch = api.FWI_STATIC_MAX_TRACES // (ns * nx) + 1
    gp, _ = problems(20, nx, 4, 50, ns, batch=batch)
    h = api.fwi_plan_create(gp, api.W2Params(n_xi=50))
    dummy = torch.zeros(1, device="cuda:0")
    with pytest.raises(api.FwiError) as e:
        api.fwi_w2_misfit_static(h, dummy, dummy, dummy, None, None)
    assert e.value.code == api.FWI_ERR_UNSUPPORTED
    assert "exceed" in str(e.value)


def test_static_scratch_limit_applies_only_without_w2(api):
    # more traces than the built-in array, but the caller takes the per-trace
    # values: the array is not used and the call matches fwi_w2_misfit
    dev = torch.device("cuda:0")
    nz, nx, nb, nt, ns = 12, 70, 4, 60, 5
    batch = api.FWI_STATIC_MAX_TRACES // (ns * nx) + 1
    gp, _ = problems(nz, nx, nb, nt, ns, batch=batch, f_peak=25.0)
    T = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    with api.Plan(gp, api.W2Params(n_xi=60)) as plan:
        vt = models("layered", list(range(batch)), nz, nx)
        v0 = models("curved_faulted", list(range(1, batch + 1)), nz, nx)
        d_obs = plan.forward(T(vt), store=False)[0].clone()
        ctx = plan.w2_prepare(d_obs)
        d_syn = plan.forward(T(v0), store=False)[0]
        J_ref, w2_ref, _ = plan.w2_misfit(ctx, d_syn)
        J = torch.empty_like(J_ref)
        w2 = torch.empty_like(w2_ref)
        api.fwi_w2_misfit_static(plan.handle, ctx, d_syn, J, w2, None)
        torch.cuda.synchronize()
        assert _rel(J, J_ref) <= TOL_J and _rel(w2, w2_ref) <= TOL_J
