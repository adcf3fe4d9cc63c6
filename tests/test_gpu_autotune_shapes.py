"""The autotuner's thread shapes on the three workload sizes: for 70 x 70 (the
resident family: column pairs or single columns), 256 x 256 (cluster strips
of 13 or 19 rows, or tiled rows) and 512 x 1024 (tiled, 8 or 4 rows a
thread, checkpointed), the (family, shape) that fwi_autotune_kernels picks
runs a whole gradient pass no slower than the default shape of the same
family, timed independently of the autotuner with CUDA events."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import initial, models, problems  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


def _pass_ms(api, prob, vt, v0, reps=3):
    with api.Plan(prob) as plan:
        d_obs, _ = plan.forward(vt, store=False)
        ctx = plan.w2_prepare(d_obs.clone())
        plan.gradient(v0, ctx)                     # untimed
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            plan.gradient(v0, ctx)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        plan.check()
    return best


@pytest.mark.parametrize("nz,nx,nb,nt,ns,batch,K", [
    (70, 70, 40, 1000, 5, 8, 0),
    (256, 256, 40, 1000, 4, 1, 0),
    (512, 1024, 40, 1000, 2, 1, 32),
])
def test_chosen_shape_is_no_slower_than_the_default(api, nz, nx, nb, nt, ns, batch, K):
    gp, _ = problems(nz, nx, nb, nt, ns, batch=batch)
    gp = dataclasses.replace(gp, checkpoint_every=K)
    vt = T(models("layered", list(range(batch)), nz, nx))
    v0 = T(initial(batch, nz, nx))
    tuned, ms = api.autotune(gp, v=v0, trial_steps=64)
    assert tuned.shape != api.SHAPE_DEFAULT        # a shape of the family is named
    default = dataclasses.replace(gp, kernels=tuned.kernels, shape=api.SHAPE_DEFAULT)
    t_tuned = _pass_ms(api, tuned, vt, v0)
    t_default = _pass_ms(api, default, vt, v0)
    print(f"{nz}x{nx}: family {tuned.kernels} shape {tuned.shape}: {t_tuned:.2f} ms, "
          f"default shape {t_default:.2f} ms, predictions {ms}")
    assert t_tuned <= 1.05 * t_default, (t_tuned, t_default, tuned.shape)
