"""Persistent passes over uneven instances (fwi_queue_forward /
fwi_queue_adjoint, api.Queue): plans of three different grid sizes, shot
counts and batches run their forward and their adjoint each as one
persistent launch, bitwise the per-plan calls; the counter is reused across
calls and graph captures."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import initial, models, problems  # noqa: E402

DEV = "cuda:0"
SIZES = [  # nz, nx, nb, ns, batch -- largest first; one physics (dx, dt, nb, source)
    (70, 70, 40, 5, 3),
    (60, 50, 40, 2, 4),
    (40, 70, 40, 3, 2),
]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def _setup(api, nt=300):
    plans, vs, ctxs = [], [], []
    for k, (nz, nx, nb, ns, B) in enumerate(SIZES):
        gp, _ = problems(nz, nx, nb, nt, ns, batch=B, f_peak=25.0)
        p = api.Plan(gp, api.W2Params(n_xi=300))
        d_obs = p.forward(T(models("curved_faulted", list(range(10 * k, 10 * k + B)), nz, nx)),
                          store=False)[0].clone()
        plans.append(p)
        ctxs.append(p.w2_prepare(d_obs))
        vs.append(T(initial(B, nz, nx)))
    return plans, vs, ctxs


def test_queue_gradient_is_bitwise_the_per_plan_gradient(api):
    plans, vs, ctxs = _setup(api)
    for p in plans:
        assert api.fwi_plan_kernels(p.handle) == api.KERNELS_RESIDENT
    ref = []
    for p, v, c in zip(plans, vs, ctxs):
        J, g, _ = p.gradient(v, c)
        ref.append((J.clone(), g.clone()))
    q = api.Queue(plans)
    for _ in range(2):                      # the counter is reset by every call
        Js, gs = q.gradient(vs, ctxs)
        torch.cuda.synchronize()
        for p in plans:
            p.check()
        for (J0, g0), J, g in zip(ref, Js, gs):
            assert torch.equal(J, J0) and torch.equal(g, g0)


def test_queue_passes_replay_from_a_graph(api):
    plans, vs, ctxs = _setup(api, nt=200)
    q = api.Queue(plans)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        q.gradient(vs, ctxs)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        Jg, gg = q.gradient(vs, ctxs)
    for seed in (1, 2):
        for v in vs:
            v.sub_(float(seed))             # new models, still inside (0, v_max]
        graph.replay()
        torch.cuda.synchronize()
        for p in plans:
            p.check()
        ref = [p.gradient(v, c) for p, v, c in zip(plans, vs, ctxs)]
        torch.cuda.synchronize()
        for (J0, g0, _), J, g in zip(ref, Jg, gg):
            assert torch.equal(J, J0) and torch.equal(g, g0)
