"""Failure detection on the GPU without a fault: the cluster and tiled
propagators' bounded halo waits run out under the self-check (every halo row
or tile withheld), the status word reports FWI_ERR_DEVICE_TIMEOUT through
fwi_check, and the device stays usable: the next forward is exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_cases import TOL_DATA, models, rel_l2  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2603_16393_gb300 import inputs as I  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


@pytest.mark.parametrize("family", ["CLUSTER", "TILED"])
def test_halo_waits_time_out_and_recover(api, family):
    nz, nx, nb, nt, ns, B = 64, 96, 20, 150, 2, 2
    geo = I.surface_geometry(nx, ns)
    kw = dict(nz=nz, nx=nx, nb=nb, nt=nt, dz=10.0, dx=10.0, dt=1e-3, src_iz=geo.src_iz,
              src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, f_peak=20.0)
    fam = getattr(api, "KERNELS_" + family)
    gp = api.Problem(**kw, batch=B, kernels=fam)
    op = O.Problem(**kw)
    v = models("layered", [1, 2], nz, nx)
    with api.Plan(gp) as plan:
        assert plan.kernels == fam
        vt = torch.tensor(v, dtype=torch.float32, device=DEV)
        d = torch.empty(plan.data_shape, dtype=torch.float32, device=DEV)
        api.fwi_forward_wait_check(plan.handle, vt, d, plan.snapshots, plan.workspace)
        torch.cuda.synchronize()
        with pytest.raises(api.FwiError) as err:
            plan.check()
        assert err.value.code == api.FWI_ERR_DEVICE_TIMEOUT
        d2, _ = plan.forward(vt)
        torch.cuda.synchronize()
        plan.check()
    assert rel_l2(d2.double().cpu().numpy(), O.forward(op, v)) <= TOL_DATA


def test_weight_gradient_wait_runs_out_and_reports():
    """The tensor-core weight gradient with every copy withheld: its bounded
    waits run out, the launch returns, the status word says so, and the next
    weight gradient on the same context is correct."""
    import numpy as np
    from paper_2603_16393_gb300 import api as A
    from oracle import score_train as T
    dev = "cuda:0"
    n, h, w, c = 1, 9, 13, 128
    rng = np.random.default_rng(21)
    x = torch.tensor(rng.standard_normal((n, h, w, c)), dtype=torch.float32).to(torch.bfloat16)
    dp = torch.tensor(rng.standard_normal((n, h, w, c)), dtype=torch.float32).to(torch.bfloat16)
    X, dP = x.to(dev), dp.to(dev)
    dW = torch.empty((c, 3, 3, c), dtype=torch.float32, device=dev)
    stage = torch.empty(A.fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, c, c), dtype=torch.uint8,
                        device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    A.fwi_conv3x3_wgrad_tc_wait_check(X, dP, dW, stage, status)
    torch.cuda.synchronize()
    assert int(status.item()) == A.FWI_ERR_DEVICE_TIMEOUT
    status.zero_()
    A.fwi_conv3x3_wgrad_tc(X, dP, dW, stage, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = T.conv3x3_wgrad(x.double().numpy(), dp.double().numpy())
    got = dW.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
