"""The learned forward surrogate trained on FD pairs, end to end on the GPU:
FD seismograms of the clean estimates that the early reverse steps produce
(70 x 70 models, 5 shots, 1000 steps) train the network, which then predicts
the FD data of held-out clean estimates far better than before training (the
gain of the trained network over an untrained one); its W2 guidance gradient
is checked against FD per noise level, and the gate of the sampler falls back
to FD when that error exceeds 5%."""
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


def test_training_on_fd_pairs_and_the_fd_gate(mods):
    A, S, SG = mods
    B, N = 128, 500
    geo = I.surface_geometry(70, 5)
    prob = A.Problem(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3, src_iz=geo.src_iz,
                     src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, v_max=4500.0,
                     batch=B)
    plan = A.Plan(prob, device=torch.device(DEV))
    prior = S.GaussianPrior.from_models(I.model_batch("curved_faulted", range(90_000, 90_064)),
                                        device=torch.device(DEV))
    betas = S.linear_betas(N, 2e-4, 0.04)
    raw = torch.tensor(I.surrogate_training_models(0, 32 * B).astype(np.float32), device=DEV)
    est = SG.early_clean_estimates(raw, prior, betas, 301, N, B, seed=1)
    v_tr, d_tr = SG.fd_pairs(plan, est)
    net = SG.ForwardSurrogate(B, 70, 70, 1000, geo.src_ix, geo.rec_ix, SG.trace_amplitude(d_tr),
                              seed=0, device=torch.device(DEV))
    # held-out: clean estimates of other models at the highest noise level
    vt = torch.tensor(I.model_batch("curved_faulted", range(5000, 5000 + B)).astype(np.float32),
                      device=DEV)
    v_ho = SG.early_clean_estimates(vt, prior, betas, N, N, B, seed=N)
    d_ho = plan.forward(v_ho, store=False)[0].clone()

    def data_err():
        d = net.forward(v_ho)
        return float((d - d_ho).norm() / d_ho.norm())

    before = data_err()
    tr = SG.SurrogateTrainer(net)
    log = SG.train(tr, v_tr, d_tr, 1600, log_every=400)
    after = data_err()
    torch.cuda.synchronize()
    plan.check()
    assert log[-1][1] < 0.1 * log[0][1] or log[-1][1] < 1e-3, log
    # what training gains: the FD data of held-out early clean estimates
    assert before > 0.5 and after < 0.05 and after < 0.1 * before, (before, after)

    # the FD gate: the surrogate's W2 gradient against FD on these models
    d_obs = plan.forward(vt, store=False)[0].clone()
    ctx = plan.w2_prepare(d_obs)
    guid = SG.SurrogateGuidance(net, plan, ctx)
    J_fd, g_fd, _ = plan.gradient(v_ho, ctx)
    g_fd = g_fd.clone()
    J_s, g_s = guid.gradient(v_ho)
    err = float(SG.rel_error(g_s, g_fd).max())
    # J through the surrogate's data is the FD J to the data error's order
    assert float(((J_s - J_fd).abs() / J_fd.abs()).max()) < 0.25
    gate = SG.GatedSurrogate(guid, threshold=0.05, check_every=5)
    _, g1 = gate.gradient(v_ho, step=N)
    assert torch.equal(g1, g_fd)                      # a check step returns the FD gradient
    assert abs(gate.records[0].error - err) < 1e-5 * max(1.0, err)
    assert gate.records[0].accepted == (err <= 0.05)
    _, g2 = gate.gradient(v_ho, step=N - 1)
    if err > 0.05:                                    # rejected: FD from here on
        assert gate.rejected and torch.equal(g2, g_fd)
    else:
        assert gate.n_surrogate == 1
