"""Checkpoint + recompute (fwi_problem.checkpoint_every = K): the forward
keeps the propagator state every K steps, and the adjoint recomputes each
K-step segment from it before running that segment backwards.

The recomputed segments run the same kernels on the same state, so data,
misfit and gradient must be bitwise identical to the store-all run.  Checked
for every propagator family (column-pair and single-column compile-time
pitch, runtime pitch), both top boundaries, K dividing nt or leaving a ragged
last segment, K = 1 and K >= nt; one case also against the oracle directly,
and the 70x70 / 5 shots / 1000 steps case at K = 32 with its memory.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_GRAD, TOL_J, initial, models, problems, rel_l2  # noqa: E402
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


def _run(api, gp, w2p, vt, v0):
    with api.Plan(gp, w2p) as plan:
        d_obs, _ = plan.forward(T(vt), store=False)
        ctx = plan.w2_prepare(d_obs.clone())
        d_syn, _ = plan.forward(T(v0))
        d_syn = d_syn.clone()
        J, g, _ = plan.gradient(T(v0), ctx)
        torch.cuda.synchronize()
        plan.check()
        return d_syn, J, g, plan.snap_bytes


@pytest.mark.parametrize("nz,nx,nb,nt,ns,top_bc,K", [
    (30, 70, 20, 300, 3, 0, 32),     # column-pair forward, ragged last segment
    (30, 70, 20, 300, 3, 0, 1),      # a checkpoint every step
    (30, 70, 20, 300, 3, 0, 300),    # one segment
    (30, 70, 20, 300, 3, 0, 1000),   # K > nt: clamped to one segment
    (41, 64, 25, 260, 2, 1, 50),     # column pairs, mirrored top
    (20, 23, 7, 300, 3, 0, 37),      # single-column fast kernels (odd padded width)
    (31, 17, 9, 250, 2, 1, 16),      # single-column, mirrored top
    (30, 126, 20, 200, 2, 0, 40),    # runtime-pitch kernels (NX = 166)
    (30, 126, 20, 200, 2, 1, 64),    # runtime pitch, mirrored top, ragged
])
def test_checkpointed_gradient_is_bitwise_the_store_all_gradient(api, nz, nx, nb, nt, ns,
                                                                 top_bc, K):
    gp, _ = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0, top_bc=top_bc)
    w2p = api.W2Params(n_xi=400)
    vt = models("layered", [7, 8], nz, nx)
    v0 = initial(2, nz, nx)
    d0, J0, g0, bytes0 = _run(api, gp, w2p, vt, v0)
    d1, J1, g1, bytes1 = _run(api, dataclasses.replace(gp, checkpoint_every=K), w2p, vt, v0)
    assert torch.equal(d0, d1)
    assert torch.equal(J0, J1)
    assert torch.equal(g0, g1), float((g0 - g1).abs().max())
    assert torch.isfinite(g1).all() and float(g1.abs().max()) > 0
    Ke = min(K, nt)
    assert bytes1 == -(-nt // Ke) * 2 * ns * 2 * gp.NZ * gp.NX * 4


def test_checkpointed_gradient_matches_oracle(api):
    nz, nx, nb, nt, ns = 24, 30, 8, 260, 3
    gp, op = problems(nz, nx, nb, nt, ns, batch=2, f_peak=25.0)
    gp = dataclasses.replace(gp, checkpoint_every=24)
    w2p, ow2 = api.W2Params(n_xi=400), O.W2Params(n_xi=400)
    vt = models("curved_faulted", [3, 4], nz, nx)
    v0 = initial(2, nz, nx)
    _, J, g, _ = _run(api, gp, w2p, vt, v0)
    octx = O.w2_prepare(O.forward(op, vt), op.dt, ow2)
    J_o, g_o, _ = O.gradient(op, v0, octx, ow2)
    assert rel_l2(J.double().cpu().numpy(), J_o) <= TOL_J * 10
    for b in range(2):
        assert rel_l2(g.double().cpu().numpy()[b], g_o[b]) <= TOL_GRAD


def test_checkpointed_full_size_bitwise_and_memory(api):
    # 16 models x 5 shots x 1000 steps, checkpoint every 32 steps
    B = 16
    gp, _ = problems(70, 70, 40, 1000, 5, batch=B)
    w2p = api.W2Params()
    vt = models("layered", list(range(B)), 70, 70)
    v0 = initial(B, 70, 70)
    _, J0, g0, bytes0 = _run(api, gp, w2p, vt, v0)
    _, J1, g1, bytes1 = _run(api, dataclasses.replace(gp, checkpoint_every=32), w2p, vt, v0)
    assert torch.equal(J0, J1) and torch.equal(g0, g1)
    # 32 checkpoints of two 110 x 150 grids per (model, shot): 4.2 MB against
    # 1000 record planes (70 MB)
    per_bs = bytes1 / (B * 5)
    assert per_bs == 32 * 2 * 110 * 150 * 4
    assert bytes0 / bytes1 > 16
