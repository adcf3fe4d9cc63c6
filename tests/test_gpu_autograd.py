"""The autograd binding: w2_fwi_objective(v).backward() against the library's
gradient entry point, the chain rule, pending forwards, and central
differences of J on the 70x70 / 5 shots / 1000 steps case with checkpoints
every 32 steps (16 models), with the device memory of both record modes.

A single cell moves J by ~1e-7 per m/s, and J is only piecewise smooth: the
interpolated quantiles change bracket so often that, along dJ/dv itself,
central differences of the FP64 objective match <dJ/dv, d> only for steps
below ~0.005 m/s -- under the float32 resolution of a velocity near 3000 m/s.
So the differences are taken on the FP64 oracle's J (h = 0.01 m/s per cell),
and the gradient under test is the GPU's.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import initial, models, problems  # noqa: E402
from oracle import oracle as O  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import autograd as G
    return A, G


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


@pytest.mark.parametrize("K", [0, 32])
def test_backward_is_the_library_gradient(mods, K):
    api, G = mods
    nz, nx, nb, nt, ns = 30, 70, 20, 300, 3
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    gp = dataclasses.replace(gp, checkpoint_every=K)
    vt = models("layered", [7, 8], nz, nx)
    v0 = initial(2, nz, nx)
    with api.Plan(gp, api.W2Params(n_xi=400)) as plan:
        d_obs, _ = plan.forward(T(vt), store=False)
        obs = plan.w2_prepare(d_obs.clone())
        J_ref, g_ref, _ = plan.gradient(T(v0), obs)
        v = T(v0).requires_grad_(True)
        J = G.w2_fwi_objective(v, plan, obs)
        J.sum().backward()
        torch.cuda.synchronize()
        assert torch.equal(J.detach(), J_ref)
        assert torch.equal(v.grad, g_ref)
        # chain rule: per-model weights scale the gradient (to the last bits:
        # a few cells of a float32 adjoint need not scale exactly even by
        # powers of two, depending on the adjoint source's bits)
        v.grad = None
        w = torch.tensor([0.5, 2.0], device=DEV)
        (w * G.w2_fwi_objective(v, plan, obs)).sum().backward()
        torch.cuda.synchronize()
        ref = g_ref * w.view(-1, 1, 1)
        assert float((v.grad - ref).abs().max()) <= 1e-6 * float(ref.abs().max())


def test_pending_forwards_keep_their_own_records(mods):
    api, G = mods
    nz, nx, nb, nt, ns = 24, 30, 8, 260, 3
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    with api.Plan(gp, api.W2Params(n_xi=400)) as plan:
        d_obs, _ = plan.forward(T(models("layered", [1, 2], nz, nx)), store=False)
        obs = plan.w2_prepare(d_obs.clone())
        va, vb = initial(2, nz, nx), models("curved_faulted", [5, 6], nz, nx) * 0.97
        _, ga, _ = plan.gradient(T(va), obs)
        ga = ga.clone()
        _, gb, _ = plan.gradient(T(vb), obs)
        ta, tb = T(va).requires_grad_(True), T(vb).requires_grad_(True)
        Ja = G.w2_fwi_objective(ta, plan, obs)
        Jb = G.w2_fwi_objective(tb, plan, obs)     # second forward before any backward
        (Ja.sum() + Jb.sum()).backward()
        torch.cuda.synchronize()
        assert torch.equal(ta.grad, ga) and torch.equal(tb.grad, gb)


def test_central_differences_with_checkpoints_full_size(mods):
    api, G = mods
    B, ns, nt = 16, 5, 1000
    gp, _ = problems(70, 70, 40, nt, ns, batch=B)
    gpk = dataclasses.replace(gp, checkpoint_every=32)
    vt = models("curved_faulted", list(range(B)), 70, 70)
    v0 = initial(B, 70, 70)
    peaks = {}
    grads = {}
    for K, prob in ((0, gp), (32, gpk)):
        with api.Plan(prob, snapshots=False) as plan:
            d_obs, _ = plan.forward(T(vt), store=False)
            obs = plan.w2_prepare(d_obs.clone())
            torch.cuda.synchronize()
            torch.cuda.reset_peak_memory_stats()
            base = torch.cuda.memory_allocated()
            v = T(v0).requires_grad_(True)
            G.w2_fwi_objective(v, plan, obs).sum().backward()
            torch.cuda.synchronize()
            peaks[K] = torch.cuda.max_memory_allocated() - base
            grads[K] = v.grad.clone()
            del d_obs
    assert torch.equal(grads[0], grads[32])
    # the record (70 MB per model and shot) against 32 checkpoints (4.2 MB)
    assert peaks[32] * 8 < peaks[0], peaks
    g = grads[32].double().cpu().numpy()

    # (i) 20 random cells among those carrying at least a tenth of their
    # model's largest gradient: central differences of the FP64 oracle's J
    # (h = 0.01 m/s, both perturbations of all 20 cells in one batch)
    rng = np.random.default_rng(2026)
    cells = []
    while len(cells) < 20:
        b, iz, ix = int(rng.integers(B)), int(rng.integers(70)), int(rng.integers(70))
        if abs(g[b, iz, ix]) >= 0.1 * np.abs(g[b]).max() and (b, iz, ix) not in cells:
            cells.append((b, iz, ix))
    h = 0.01
    vp = np.stack([v0[b] for b, _, _ in cells for _ in (0, 1)])
    for k, (b, iz, ix) in enumerate(cells):
        vp[2 * k, iz, ix] += h
        vp[2 * k + 1, iz, ix] -= h
    _, op = problems(70, 70, 40, nt, ns, batch=1)
    ow2 = O.W2Params()
    octx = O.w2_prepare(O.forward(op, np.stack([vt[b] for b, _, _ in cells for _ in (0, 1)])),
                        op.dt, ow2)
    J_o = O.w2_misfit(octx, O.forward(op, vp), op.dt, ow2, with_adjoint=False)[0]
    fd = (J_o[0::2] - J_o[1::2]) / (2 * h)
    an = np.array([g[b, iz, ix] for b, iz, ix in cells])
    scale = np.array([np.abs(g[b]).max() for b, _, _ in cells])
    assert np.all(np.abs(fd - an) <= 2e-3 * scale), np.abs(fd - an) / scale
