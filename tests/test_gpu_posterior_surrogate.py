"""Algorithm 2 on noisy observations with the trained forward surrogate in the
first 40% of the reverse steps, against the same chain with FD guidance in
every step (70 x 70 models, 5 shots x 1000 FD steps, 10 dB observations, 2
observations x 15 posterior samples, 100 reverse steps):
  * gated at 5% (the FD solver as the check): the first check rejects the
    surrogate (its W2 gradient misses FD's by far more than 5% on these
    inputs) and the chain falls back to FD for good -- bitwise the FD chain;
  * used without the gate: the chain costs at most 0.8 of the FD chain and
    its samples reconstruct the true models as well (RMSE within 2%): in the
    high-noise steps the chain rule scales the guidance by sqrt(abar_i), so
    the surrogate's error there barely reaches the samples, while its cost
    replaces 40% of the FD solves."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_16393_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    from paper_2603_16393_gb300 import sampler as S
    from paper_2603_16393_gb300 import surrogate as SG
    return A, S, SG


def test_surrogate_phase_cost_and_reconstruction(mods):
    A, S, SG = mods
    n_obs, P, N = 2, 15, 100
    B = n_obs * P
    geo = I.surface_geometry(70, 5)
    prob = A.Problem(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3, src_iz=geo.src_iz,
                     src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, v_max=4500.0,
                     batch=B)
    dev = torch.device(DEV)
    plan = A.Plan(prob, device=dev)
    vt = I.model_batch("curved_faulted", range(7000, 7000 + n_obs))
    vt_rep = np.repeat(vt, P, axis=0)
    vt_d = torch.tensor(vt_rep, dtype=torch.float32, device=DEV)
    d_clean = plan.forward(vt_d, store=False)[0].cpu().numpy()
    noise = np.concatenate([np.repeat(I.gaussian_noise_like(d_clean[o * P:o * P + 1], 10.0,
                                                            7000 + o), P, axis=0)
                            for o in range(n_obs)])
    ctx = plan.w2_prepare(torch.tensor(d_clean + noise, dtype=torch.float32, device=DEV))
    prior = S.GaussianPrior.from_models(I.model_batch("curved_faulted", range(90_000, 90_064)),
                                        device=dev)
    betas = S.linear_betas(N, 1e-4 * 1000 / N, 0.02 * 1000 / N)
    guide = A.GuideParams(rho0=100.0, gamma=0.55, c=1e9)
    gen = torch.Generator(device=DEV).manual_seed(4321)
    zs = torch.randn((N + 1, B, 70, 70), device=DEV, generator=gen)
    v_start = torch.randn((B, 70, 70), device=DEV, generator=gen)

    # the surrogate, trained on FD pairs of clean estimates of its 40 steps
    # (minibatches of 32 models, four full images of 8), then given to a
    # network of the chain's 30 models
    i_switch = N - 40
    BT = 32
    plan_t = A.Plan(dataclasses.replace(prob, batch=BT), device=dev)
    raw = torch.tensor(I.surrogate_training_models(0, 64 * BT).astype(np.float32), device=DEV)
    est = SG.early_clean_estimates(raw, prior, betas, i_switch + 1, N, BT, seed=1)
    v_tr, d_tr = SG.fd_pairs(plan_t, est)
    amp = SG.trace_amplitude(d_tr)
    net_t = SG.ForwardSurrogate(BT, 70, 70, 1000, geo.src_ix, geo.rec_ix, amp, seed=0, device=dev)
    tr = SG.SurrogateTrainer(net_t)
    SG.train(tr, v_tr, d_tr, 1200)
    tr.lr = 3e-4
    SG.train(tr, v_tr, d_tr, 600)
    net = SG.ForwardSurrogate(B, 70, 70, 1000, geo.src_ix, geo.rec_ix, amp, seed=0, device=dev)
    SG.copy_weights(net, net_t)
    guid = SG.SurrogateGuidance(net, plan, ctx)

    def timed_run(chain):
        chain.run(v_start, N, N - 1)                # captures and warm replays
        torch.cuda.synchronize()
        chain.counts = {k: 0 for k in chain.counts}
        chain.records.clear()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        v = chain.run(v_start).clone()
        b.record()
        torch.cuda.synchronize()
        return v, a.elapsed_time(b)

    def rmse(x):
        v = (3000.0 + 1500.0 * x).clamp(1500.0, 4500.0)
        return float(((v - vt_d) ** 2).mean().sqrt())

    fd = S.GraphChain(plan, betas, ctx, prior, guide, zs)
    v_fd, ms_fd = timed_run(fd)
    gated = S.GraphChain(plan, betas, ctx, prior, guide, zs, surrogate=guid,
                         surrogate_fraction=0.4, threshold=0.05, check_every=10)
    v_gated, _ = timed_run(gated)
    free = S.GraphChain(plan, betas, ctx, prior, guide, zs, surrogate=guid,
                        surrogate_fraction=0.4, threshold=float("inf"), check_every=10)
    v_free, ms_free = timed_run(free)
    plan.check()

    # gated: the FD check's first verdict decides the chain
    first = gated.records[0]
    if not first[2]:
        assert gated.counts["sur"] == 0
        assert torch.equal(v_gated, v_fd)       # FD fallback: the FD chain, bit for bit
    # ungated: 36 surrogate steps, 4 checks, 60 FD steps
    assert free.counts == {"fd": 60, "sur": 36, "check": 4}, free.counts
    r_fd, r_free = rmse(v_fd), rmse(v_free)
    assert ms_free < 0.8 * ms_fd, (ms_free, ms_fd)
    assert abs(r_free - r_fd) < 0.02 * r_fd, (r_free, r_fd)
