"""The batched and large-grid workloads, checked on the GPU:

  * 64 curved/faulted 70 x 70 models, 5 shots, 1000 steps, observed data with
    10 dB SNR Gaussian noise (sigma^2 = mean(d^2) / 10 per instance);
  * 8 models of 256 x 256, 16 shots, 2000 steps (cluster kernels);
  * 2 models of 512 x 1024 (depth x width), 32 shots, 4000 steps, with
    checkpoints every 32 steps (the whole wavefield record would need 624 GB).

Sampled instances are compared with the FP64 oracle on the same inputs (the
noisy observations are the oracle's clean data plus seeded noise, rounded to
float32, handed to both sides).  The 512 x 1024 run is checked by properties
that hold at any size (finite outputs; checkpoint interval and batch
composition change no bit of J or dJ/dv), and one of its shots against the
oracle over the whole 4000 steps.

End-to-end parity of dJ/dv on the long runs (256 x 256 / 2000 steps, 512 x
1024 / 4000 steps): the W2 misfit's quantile map amplifies data errors where a
CDF crosses xi_j at low density, so a float32 forward's data error (a few
1e-7 RMS there; 1e-5 is the bar) moves the FP64 objective's own gradient by
more than 1e-4.  The end-to-end bar on those runs is therefore an envelope
measured in the test itself: the spread of the oracle's gradient when its own
synthetic data carry white noise as large as the GPU's measured data error;
the GPU gradient must lie within a few of those spreads.  The stages keep the
usual bars on their own (forward data 1e-5, adjoint on a shared adjoint source
1e-4).
"""
import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_DATA, TOL_GRAD, TOL_J, initial, models, problems, rel_l2  # noqa: E402
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


def test_64_curved_models_with_10db_noise(api):
    B, ns, nt = 64, 5, 1000
    gp, op = problems(70, 70, 40, nt, ns, batch=B)
    vt = models("curved_faulted", list(range(B)), 70, 70)
    v0 = initial(B, 70, 70)
    clean = O.forward(op, vt)
    d_obs = clean + I.gaussian_noise_like(clean, 10.0, seed=10)
    d_obs = d_obs.astype(np.float32).astype(np.float64)
    with api.Plan(gp) as plan:
        ctx = plan.w2_prepare(T(d_obs))
        J, g, _ = plan.gradient(T(v0), ctx)
        torch.cuda.synchronize()
        plan.check()
    ow2 = O.W2Params()
    for b in (0, 31, 63):
        octx = O.w2_prepare(d_obs[b:b + 1], op.dt, ow2)
        J_o, g_o, _ = O.gradient(op, v0[b:b + 1], octx, ow2)
        assert abs(float(J[b]) - J_o[0]) <= TOL_J * 10 * abs(J_o[0]), (b, float(J[b]), J_o[0])
        assert rel_l2(H(g)[b], g_o[0]) <= TOL_GRAD, (b, rel_l2(H(g)[b], g_o[0]))


ENVELOPE = 4.0     # GPU error <= ENVELOPE x the oracle's spread (see the module docstring)


def _oracle_envelope(op, v, octx, ow2, g_o, data_err, seeds=(1, 2)):
    """The largest rel-L2 change of the oracle's gradient at v when its
    synthetic data carry white noise of relative RMS data_err."""
    d = O.forward(op, v[None])
    rms = float(np.sqrt(np.mean(d * d)))
    out = 0.0
    for sd in seeds:
        noise = data_err * rms * np.random.default_rng(sd).standard_normal(d.shape)
        _, _, adj = O.w2_misfit(octx, d + noise, op.dt, ow2)
        out = max(out, rel_l2(_oracle_adjoint_stage(op, v, adj[0]), g_o))
    return out


def _oracle_adjoint_stage(op, v, adj):
    """dJ/dv of one model for a given adjoint source [ns][nr][nt] (FP64)."""
    def unit(s):
        _, u_all = O.forward_shot(op, v, s, keep_wavefield=True)
        return O.fold(op, O.adjoint_shot(op, v, s, adj[s], u_all))
    with ThreadPoolExecutor(O.nthreads()) as ex:
        return sum(ex.map(unit, range(op.ns)))


def test_8_models_256x256_16_shots_2000_steps(api):
    B, ns, nt, n = 8, 16, 2000, 256
    gp, op = problems(n, n, 40, nt, ns, batch=B)
    vt = models("curved_faulted", list(range(B)), n, n)
    v0 = initial(B, n, n)
    b_s = 5
    adj = np.random.default_rng(0).standard_normal((B, ns, gp.nr, nt))
    adj = adj.astype(np.float32).astype(np.float64)
    with api.Plan(gp) as plan:
        assert plan.kernels == api.KERNELS_CLUSTER      # 296 x 336 cells: 8 CTAs of 38 rows
        d_obs, _ = plan.forward(T(vt), store=False)
        d_obs = d_obs.clone()
        # the sampled instance observes the oracle's data
        d_o = O.forward(op, vt[b_s:b_s + 1]).astype(np.float32).astype(np.float64)
        d_obs[b_s] = T(d_o[0])
        ctx = plan.w2_prepare(d_obs)
        J, g, _ = plan.gradient(T(v0), ctx)
        J, g = H(J), H(g)
        d_syn = H(plan.forward(T(v0))[0])
        g_adj = H(plan.adjoint_grad(T(v0), T(adj)))   # adjoint stage on a shared source
        torch.cuda.synchronize()
        plan.check()
    assert np.isfinite(g).all() and np.isfinite(J).all()
    # each stage at its own bar
    data_err = rel_l2(d_syn[b_s], O.forward(op, v0[b_s:b_s + 1])[0])
    assert data_err <= TOL_DATA
    assert rel_l2(g_adj[b_s], _oracle_adjoint_stage(op, v0[b_s], adj[b_s])) <= TOL_GRAD
    # end to end, within the oracle's own envelope at that data error
    ow2 = O.W2Params()
    octx = O.w2_prepare(d_o, op.dt, ow2)
    J_o, g_o, _ = O.gradient(op, v0[b_s:b_s + 1], octx, ow2)
    assert abs(J[b_s] - J_o[0]) <= TOL_J * 10 * abs(J_o[0]), (J[b_s], J_o[0])
    spread = _oracle_envelope(op, v0[b_s], octx, ow2, g_o[0], data_err)
    err = rel_l2(g[b_s], g_o[0])
    assert err <= max(ENVELOPE * spread, TOL_GRAD), (err, spread, data_err)


def test_512x1024_grid_against_the_oracle_over_600_steps(api):
    nz, nx, ns, nt = 512, 1024, 8, 600
    gp, op = problems(nz, nx, 40, nt, ns, batch=1)
    vt = models("curved_faulted", [3], nz, nx)
    v0 = initial(1, nz, nx)
    d_o = O.forward(op, vt).astype(np.float32).astype(np.float64)
    with api.Plan(dataclasses.replace(gp, checkpoint_every=32)) as plan:
        ctx = plan.w2_prepare(T(d_o))
        J, g, _ = plan.gradient(T(v0), ctx)
        torch.cuda.synchronize()
        plan.check()
    ow2 = O.W2Params()
    octx = O.w2_prepare(d_o, op.dt, ow2)
    J_o, g_o, _ = O.gradient(op, v0, octx, ow2)
    assert abs(float(J[0]) - J_o[0]) <= TOL_J * 10 * abs(J_o[0]), (float(J[0]), J_o[0])
    assert rel_l2(H(g)[0], g_o[0]) <= TOL_GRAD, rel_l2(H(g)[0], g_o[0])


def test_2_models_512x1024_32_shots_4000_steps_checkpointed(api):
    # properties that hold at any size: checkpoint interval and batch
    # composition do not change a single bit of J or dJ/dv
    B, ns, nt, nz, nx = 2, 32, 4000, 512, 1024
    gp, _ = problems(nz, nx, 40, nt, ns, batch=B)
    vt = models("curved_faulted", [0, 1], nz, nx)
    v0 = initial(B, nz, nx)
    out = {}
    for K, b in ((32, B), (64, B), (32, 1)):
        prob = dataclasses.replace(gp, checkpoint_every=K, batch=b)
        with api.Plan(prob) as plan:
            if (K, b) == (32, B):
                assert plan.snap_bytes == 125 * B * ns * 2 * 552 * 1104 * 4
            d_obs, _ = plan.forward(T(vt[B - b:]), store=False)
            ctx = plan.w2_prepare(d_obs.clone())
            J, g, _ = plan.gradient(T(v0[B - b:]), ctx)
            torch.cuda.synchronize()
            plan.check()
            out[(K, b)] = (J.clone(), g.clone())
    J, g = out[(32, B)]
    assert torch.isfinite(g).all() and torch.isfinite(J).all()
    assert float(g.abs().max()) > 0 and float(J.min()) > 0
    assert torch.equal(J, out[(64, B)][0]) and torch.equal(g, out[(64, B)][1])
    assert torch.equal(J[1:], out[(32, 1)][0]) and torch.equal(g[1:], out[(32, 1)][1])


def test_512x1024_one_shot_4000_steps_against_the_oracle(api):
    # the whole time axis of the 512 x 1024 workload for one model and one
    # shot (the oracle keeps every wavefield level: 19.5 GB in FP64)
    nz, nx, ns, nt = 512, 1024, 1, 4000
    geo = I.surface_geometry(nx, 1)
    gp, op = problems(nz, nx, 40, nt, ns, batch=1, geo=geo)
    vt = models("curved_faulted", [4], nz, nx)
    v0 = initial(1, nz, nx)
    d_o = O.forward(op, vt).astype(np.float32).astype(np.float64)
    with api.Plan(dataclasses.replace(gp, checkpoint_every=32)) as plan:
        ctx = plan.w2_prepare(T(d_o))
        J, g, _ = plan.gradient(T(v0), ctx)
        d_syn = H(plan.forward(T(v0), store=False)[0])
        torch.cuda.synchronize()
        plan.check()
    data_err = rel_l2(d_syn[0], O.forward(op, v0)[0])
    assert data_err <= TOL_DATA
    ow2 = O.W2Params()
    octx = O.w2_prepare(d_o, op.dt, ow2)
    J_o, g_o, _ = O.gradient(op, v0, octx, ow2)
    assert abs(float(J[0]) - J_o[0]) <= TOL_J * 10 * abs(J_o[0]), (float(J[0]), J_o[0])
    spread = _oracle_envelope(op, v0[0], octx, ow2, g_o[0], data_err, seeds=(1,))
    err = rel_l2(H(g)[0], g_o[0])
    assert err <= max(ENVELOPE * spread, TOL_GRAD), (err, spread, data_err)
