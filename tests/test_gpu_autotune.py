"""GPU checks of the kernel-family autotuner: it times every family that can
run a problem, picks the fastest, and the plan made with its choice gives
the same gradient as the automatic choice (float rounding apart)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import initial, models, problems, rel_l2  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device=DEV)


@pytest.mark.parametrize("nz,nx,nb,n_fam", [
    (30, 70, 20, 3),      # 50 x 110 cells: resident, tiled and cluster all run it
    (100, 140, 20, 2),    # 120 x 180 cells: beyond one CTA
])
def test_autotune_times_every_family_and_picks_the_fastest(api, nz, nx, nb, n_fam):
    gp, _ = problems(nz, nx, nb, 300, 3, batch=2, f_peak=25.0)
    v = T(initial(2, nz, nx))
    n = api.fwi_autotune_scratch_bytes(gp, api.W2Params(), 40)
    scratch = torch.empty(n, dtype=torch.uint8, device=DEV)
    fams = [api.KERNELS_RESIDENT, api.KERNELS_TILED, api.KERNELS_CLUSTER, api.KERNELS_CPML]
    family_shapes = {api.KERNELS_RESIDENT: (api.SHAPE_RESIDENT_PAIRS, api.SHAPE_RESIDENT_COLUMNS),
                     api.KERNELS_TILED: (api.SHAPE_TILED_ROWS8, api.SHAPE_TILED_ROWS4,
                                         api.SHAPE_TILED_QUADS),
                     api.KERNELS_CLUSTER: (api.SHAPE_CLUSTER_PAIRS, api.SHAPE_CLUSTER_RS13,
                                           api.SHAPE_CLUSTER_RS19)}
    for _ in range(2):                      # twice in a row on the same scratch
        fam, shape, ms, shapes = api.fwi_autotune_kernels(gp, api.W2Params(), v, 40, scratch)
        ran = [t for t in ms if t >= 0]
        assert len(ran) == n_fam and all(t > 0 for t in ran)
        assert len(ms) == 4 and ms[3] == -1 and shapes[3] == -1   # CPML: CPML problems only
        assert ms[fams.index(fam)] == min(ran)
        # every family that ran names one of its own shapes, the chosen one too
        for f, t, sh in zip(fams[:3], ms, shapes):
            assert (t < 0 and sh == -1) or sh in family_shapes[f]
        assert shape == shapes[fams.index(fam)]
    # the scratch must cover the trial plans
    with pytest.raises(api.FwiError) as e:
        api.fwi_autotune_kernels(gp, api.W2Params(), v, 40, scratch[: n // 2])
    assert e.value.code == 6


def test_autotuned_plan_gives_the_automatic_gradient(api):
    nz, nx, nb = 100, 140, 20
    gp, _ = problems(nz, nx, nb, 300, 2, batch=2, f_peak=25.0)
    tuned, ms = api.autotune(gp, trial_steps=32)
    assert tuned.kernels in (api.KERNELS_TILED, api.KERNELS_CLUSTER) and ms[0] == -1
    w2p = api.W2Params(n_xi=400)
    vt, v0 = T(models("layered", [1, 2], nz, nx)), T(initial(2, nz, nx))
    out = []
    for prob in (gp, tuned):
        with api.Plan(prob, w2p) as plan:
            d_obs, _ = plan.forward(vt, store=False)
            J, g, _ = plan.gradient(v0, plan.w2_prepare(d_obs.clone()))
            torch.cuda.synchronize()
            plan.check()
            out.append((J.double().cpu().numpy(), g.double().cpu().numpy()))
    assert rel_l2(out[1][0], out[0][0]) <= 1e-4
    for b in range(2):
        assert rel_l2(out[1][1][b], out[0][1][b]) <= 1e-3
