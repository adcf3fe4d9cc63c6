"""A whole gradient (forward, misfit, adjoint; for the tiled kernels one
launch per time step) captured once into a CUDA graph and replayed on new
models: bitwise the eager result, for the resident, the tiled, the cluster
and the checkpointed paths.
"""
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


@pytest.mark.parametrize("nz,nx,nb,nt,ns,K,fam", [
    (30, 70, 20, 300, 3, 0, 0),       # shared-memory resident kernels
    (100, 140, 20, 200, 2, 0, 2),     # tiled kernels, one launch per step
    (100, 140, 20, 200, 2, 0, 3),     # cluster kernels
    (100, 140, 20, 200, 2, 64, 0),    # tiled, checkpointed
    (30, 70, 20, 300, 3, 32, 0),      # resident, checkpointed
])
def test_gradient_replays_from_a_cuda_graph(api, nz, nx, nb, nt, ns, K, fam):
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, v_max=4600.0)
    gp = dataclasses.replace(gp, checkpoint_every=K, kernels=fam)
    plan = api.Plan(gp, api.W2Params(n_xi=400))
    d_obs, _ = plan.forward(T(models("layered", [1, 2], nz, nx)), store=False)
    ctx = plan.w2_prepare(d_obs.clone())
    v_static = T(initial(2, nz, nx))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):                       # warm-up outside the capture
            plan.gradient(v_static, ctx)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        J_g, g_g, _ = plan.gradient(v_static, ctx)
    for seed in (3, 4):
        v_new = initial(2, nz, nx) + np.stack([I.smooth_perturbation(seed + b, nz, nx, 50.0)
                                               for b in range(2)])
        v_static.copy_(T(v_new))
        graph.replay()
        J_e, g_e, _ = plan.gradient(T(v_new), ctx)
        torch.cuda.synchronize()
        plan.check()
        assert torch.equal(J_g, J_e) and torch.equal(g_g, g_e)
        assert float(g_e.abs().max()) > 0
