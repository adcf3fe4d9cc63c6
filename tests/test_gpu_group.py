"""Plan groups (fwi_group_gradient): uneven instances -- a shared-memory
resident grid, a cluster grid and a tiled, checkpointed grid -- run as one
unit on forked streams, with results bitwise those of the per-plan calls,
and the whole set captured into one CUDA graph and replayed on new models."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import initial, models, problems  # noqa: E402
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


def _members(api):
    cases = [(30, 70, 20, 300, 3, 2, {}),                                  # resident
             (100, 140, 20, 200, 2, 1, {}),                                # cluster
             (40, 260, 10, 200, 2, 1, dict(kernels=2, checkpoint_every=48))]  # tiled, checkpoints
    out = []
    for nz, nx, nb, nt, ns, B, kw in cases:
        gp, _ = problems(nz, nx, nb, nt, ns, batch=B, f_peak=25.0, v_max=4600.0)
        plan = api.Plan(dataclasses.replace(gp, **kw), api.W2Params(n_xi=300))
        d_obs, _ = plan.forward(T(models("curved_faulted", list(range(B)), nz, nx)), store=False)
        ctx = plan.w2_prepare(d_obs.clone())
        out.append((plan, ctx, (B, nz, nx)))
    return out


def test_group_gradient_is_the_per_plan_gradient(api):
    members = _members(api)
    assert [m[0].kernels for m in members] == [api.KERNELS_RESIDENT, api.KERNELS_CLUSTER,
                                                api.KERNELS_TILED]
    vs = [T(initial(*shape)) for _, _, shape in members]
    group = api.Group([m[0] for m in members])
    Jg, gg = group.gradient(vs, [m[1] for m in members])
    torch.cuda.synchronize()
    for (plan, ctx, _), v, J, g in zip(members, vs, Jg, gg):
        plan.check()
        J1, g1, _ = plan.gradient(v, ctx)
        torch.cuda.synchronize()
        assert torch.equal(J, J1) and torch.equal(g, g1)
        assert float(g.abs().max()) > 0
    group.close()


def test_group_replays_from_one_cuda_graph(api):
    members = _members(api)
    group = api.Group([m[0] for m in members])
    ctxs = [m[1] for m in members]
    vs = [T(initial(*shape)) for _, _, shape in members]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            group.gradient(vs, ctxs)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        Jg, gg = group.gradient(vs, ctxs)
    for seed in (5, 6):
        for v, (_, _, (B, nz, nx)) in zip(vs, members):
            v.copy_(T(initial(B, nz, nx) + np.stack([I.smooth_perturbation(seed + b, nz, nx, 40.0)
                                                     for b in range(B)])))
        graph.replay()
        torch.cuda.synchronize()
        Jr = [J.clone() for J in Jg]
        gr = [g.clone() for g in gg]
        Je, ge = group.gradient(vs, ctxs)
        torch.cuda.synchronize()
        for a, b in zip(Jr + gr, Je + ge):
            assert torch.equal(a, b)
    for plan, _, _ in members:
        plan.check()
    group.close()
