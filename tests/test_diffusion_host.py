"""Reverse-diffusion entry points on the host (no GPU): the per-step
coefficients of Algorithms 1-2 that fwi_ddpm_coefficients forms in FP64
agree with the oracle's schedule, and the elementwise calls reject bad
arguments before any CUDA call."""
import ctypes
import math

import numpy as np
import pytest

from oracle import diffusion as D


@pytest.fixture(scope="module")
def api():
    from paper_2603_16393_gb300 import api as A
    return A


@pytest.mark.parametrize("mode,name", [(0, "posterior"), (1, "beta")])
def test_coefficients_match_the_oracle_schedule(api, mode, name):
    betas = D.linear_betas(1000)
    sched = D.Schedule(betas, sigma=name)
    for i in (1, 2, 3, 17, 250, 999, 1000):
        st = api.fwi_ddpm_coefficients(list(betas), i, mode)
        c_v, c_0, sg = sched.proposal_coefficients(i)
        assert math.isclose(st.abar, sched.abar[i], rel_tol=1e-14)
        assert math.isclose(st.c_v, c_v, rel_tol=1e-12, abs_tol=1e-300)
        assert math.isclose(st.c_0, c_0, rel_tol=1e-12)
        assert math.isclose(st.sigma, sg, rel_tol=1e-12, abs_tol=1e-300)


def test_coefficients_of_a_cosine_like_schedule(api):
    # any schedule in (0, 1): abar is the product of the alphas up to i
    rng = np.random.default_rng(2)
    betas = np.sort(rng.uniform(1e-5, 0.3, 64))
    sched = D.Schedule(betas)
    for i in (1, 8, 64):
        st = api.fwi_ddpm_coefficients(list(betas), i)
        assert math.isclose(st.abar, sched.abar[i], rel_tol=1e-13)
        assert math.isclose(st.c_0, sched.proposal_coefficients(i)[1], rel_tol=1e-12)


def test_coefficients_reject_bad_arguments(api):
    lib = api._lib
    out = api._DdpmStep()
    b = (ctypes.c_double * 3)(0.1, 0.2, 0.3)
    bad = (ctypes.c_double * 3)(0.1, 1.0, 0.3)
    assert lib.fwi_ddpm_coefficients(None, 3, 1, 0, ctypes.byref(out)) == 1
    assert lib.fwi_ddpm_coefficients(b, 3, 1, 0, None) == 1
    assert lib.fwi_ddpm_coefficients(b, 3, 0, 0, ctypes.byref(out)) == 1
    assert lib.fwi_ddpm_coefficients(b, 3, 4, 0, ctypes.byref(out)) == 1
    assert lib.fwi_ddpm_coefficients(b, 3, 1, 2, ctypes.byref(out)) == 1
    assert lib.fwi_ddpm_coefficients(bad, 3, 2, 0, ctypes.byref(out)) == 1
    assert lib.fwi_ddpm_coefficients(bad, 3, 1, 0, ctypes.byref(out)) == 0   # only beta_1 is read
    with pytest.raises(api.FwiError):
        api.fwi_ddpm_coefficients([0.1, -0.2], 2)


def test_elementwise_calls_reject_bad_arguments_without_a_gpu(api):
    lib = api._lib
    st = api._DdpmStep(0.5, 0.3, 0.6, 0.1)
    sp = api._Space(3000.0, 1500.0, 1500.0, 4500.0)
    x = ctypes.c_void_p(16)   # never dereferenced: every call below fails its host checks
    S, P = ctypes.byref(st), ctypes.byref(sp)
    calls = [
        lambda: lib.fwi_ddpm_proposal(0, 4, S, P, x, x, x, x, x, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 0, S, P, x, x, x, x, x, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 4, None, P, x, x, x, x, x, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 4, S, None, x, x, x, x, x, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 4, S, P, None, x, x, x, x, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 4, S, P, x, None, None, x, x, x, x, x, None),  # no mu
        lambda: lib.fwi_ddpm_proposal(1, 4, S, P, x, x, x, x, None, x, x, x, None),
        lambda: lib.fwi_ddpm_proposal(1, 4, S, P, x, x, x, x, x, x, None, x, None),
        lambda: lib.fwi_ddpm_guidance(1, 4, S, P, None, x, None, None, x, x, None),
        lambda: lib.fwi_ddpm_guidance(1, 4, S, P, x, x, None, None, x, None, None),
        lambda: lib.fwi_ddpm_guidance(-1, 4, S, P, x, x, None, None, x, x, None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, k
        assert api.fwi_last_error() != ""
    for bad_step in (api._DdpmStep(0.0, 0.3, 0.6, 0.1), api._DdpmStep(1.5, 0.3, 0.6, 0.1),
                     api._DdpmStep(0.5, math.nan, 0.6, 0.1), api._DdpmStep(0.5, 0.3, 0.6, -1.0)):
        assert lib.fwi_ddpm_guidance(1, 4, ctypes.byref(bad_step), P, x, x, None, None, x, x,
                                     None) == 1
    for bad_space in (api._Space(3000.0, 0.0, 1500.0, 4500.0),
                      api._Space(3000.0, 1500.0, 4500.0, 1500.0),
                      api._Space(math.inf, 1500.0, 1500.0, 4500.0)):
        assert lib.fwi_ddpm_guidance(1, 4, S, ctypes.byref(bad_space), x, x, None, None, x, x,
                                     None) == 1


def test_conv_rejects_bad_arguments_without_a_gpu(api):
    lib = api._lib
    p = ctypes.c_void_p(4096)          # never dereferenced: every call fails its host checks
    odd = ctypes.c_void_p(4096 + 8)
    calls = [
        lambda: lib.fwi_conv3x3_bf16(0, 4, 4, 64, 64, p, p, None, 0, p, 0, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 32, 64, p, p, None, 0, p, 0, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 64, 96, p, p, None, 0, p, 0, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 64, 64, None, p, None, 0, p, 0, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 64, 64, p, p, None, 2, p, 0, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 64, 64, p, p, None, 0, p, 3, None, None),
        lambda: lib.fwi_conv3x3_bf16(1, 4, 4, 64, 64, odd, p, None, 0, p, 0, None, None),
        # the fused pre-activation + SiLU layer: no activation output, a
        # misaligned one, no pre-activation output, an empty batch
        lambda: lib.fwi_conv3x3_bf16_silu(1, 4, 4, 64, 64, p, p, None, p, None, None, None),
        lambda: lib.fwi_conv3x3_bf16_silu(1, 4, 4, 64, 64, p, p, None, p, odd, None, None),
        lambda: lib.fwi_conv3x3_bf16_silu(1, 4, 4, 64, 64, p, p, None, None, p, None, None),
        lambda: lib.fwi_conv3x3_bf16_silu(0, 4, 4, 64, 64, p, p, None, p, p, None, None),
        # the gradient convolution times SiLU': no pre-activation, a misaligned one
        lambda: lib.fwi_conv3x3_bf16_silu_grad(1, 4, 4, 64, 64, p, p, None, p, None, None),
        lambda: lib.fwi_conv3x3_bf16_silu_grad(1, 4, 4, 64, 64, p, p, odd, p, None, None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, k
        assert api.fwi_last_error() != ""


def test_grid_transfers_reject_bad_arguments_without_a_gpu(api):
    lib = api._lib
    p = ctypes.c_void_p(4096)
    calls = [
        lambda: lib.fwi_restrict2(0, 4, 4, p, p, None),
        lambda: lib.fwi_restrict2(1, 4, 4, None, p, None),
        lambda: lib.fwi_restrict2_transpose(1, 0, 4, p, p, None),
        lambda: lib.fwi_restrict2_transpose(1, 4, 4, p, None, None),
        lambda: lib.fwi_decimate2(1, 1, 1, 1, p, p, None),
        lambda: lib.fwi_decimate2(1, 1, 2, 4, None, p, None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, k
        assert api.fwi_last_error() != ""


def test_training_calls_reject_bad_arguments_without_a_gpu(api):
    lib = api._lib
    p = ctypes.c_void_p(4096)
    calls = [
        lambda: lib.fwi_dsm_noisy(4, 1.0, p, p, p, None),             # abar must be < 1
        lambda: lib.fwi_dsm_noisy(4, 0.5, None, p, p, None),
        lambda: lib.fwi_dsm_loss(0, p, p, p, p, None, 0, None),
        lambda: lib.fwi_conv3x3_wgrad(1, 4, 4, 96, 64, p, p, p, None, 0, None),   # cin % 64
        lambda: lib.fwi_conv3x3_wgrad(1, 4, 4, 64, 64, p, None, p, None, 0, None),
        lambda: lib.fwi_conv3x3_wgrad(1, 4, 4, 64, 64, ctypes.c_void_p(4100), p, p, None, 0, None),
        lambda: lib.fwi_conv3x3_wgrad_tc(1, 4, 4, 96, 128, p, p, p, p, 1 << 20, None, 0, None,
                                         None),                          # cin % 64
        lambda: lib.fwi_conv3x3_wgrad_tc(1, 4, 4, 128, 128, p, p, p, p, 16, None, 0, None,
                                         None),                          # stage too small
        lambda: lib.fwi_pool2_bf16(1, 4, 4, 12, 0, p, p, None),           # channels % 8
        lambda: lib.fwi_pool2_bf16(1, 4, 4, 16, 2, p, p, None),           # mode
        lambda: lib.fwi_up2_bf16(1, 4, 4, 16, 0, ctypes.c_void_p(4100), p, None),
        lambda: lib.fwi_add_bf16(12, p, p, p, None),
        lambda: lib.fwi_channel_sum(16, 0, p, p, None, 0, None),
        lambda: lib.fwi_adam_step(8, 1e-3, 0.9, 0.999, 1e-8, 0, p, p, p, p, None),   # step >= 1
        lambda: lib.fwi_adam_step(8, 1e-3, 1.0, 0.999, 1e-8, 1, p, p, p, p, None),
        lambda: lib.fwi_adam_step(8, 0.0, 0.9, 0.999, 1e-8, 1, p, p, p, p, None),
        lambda: lib.fwi_conv3x3_weights_prep(64, 64, p, None, p, None),
        lambda: lib.fwi_time_bias(0, 64, 16, p, p, p, p, None),
        lambda: lib.fwi_time_bias_grad(64, 16, p, None, p, None),
    ]
    for k, call in enumerate(calls):
        assert call() == 1, k
        assert api.fwi_last_error() != ""
    # the split count: 1 without room for a second range, at most 16
    assert lib.fwi_conv3x3_wgrad_splits(2, 33, 47, 64, 64, 0) == 1
    assert lib.fwi_conv3x3_wgrad_splits(2, 33, 47, 64, 64, 9 * 64 * 64 * 3) in (2, 3)
    assert 1 <= lib.fwi_conv3x3_wgrad_splits(152, 70, 70, 128, 128, 10 ** 9) <= 16
    assert lib.fwi_conv3x3_wgrad_splits(1, 4, 4, 96, 64, 10 ** 9) == 0
    # the tensor-core staging buffer: (cout + 3 cin) x padded pixels x 2 bytes
    wp = 72
    assert lib.fwi_conv3x3_wgrad_tc_stage_bytes(152, 70, 70, 128, 256) == \
        (256 + 3 * 128) * 152 * 72 * wp * 2
    assert lib.fwi_conv3x3_wgrad_tc_stage_bytes(1, 4, 4, 96, 128) == 0
    assert lib.fwi_conv3x3_wgrad_tc_stage_bytes(1, 4, 4, 64, 128) == (128 + 3 * 64) * 6 * 8 * 2


def test_coarse_problem_of_the_benchmark(api):
    prob = api.Problem(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3,
                       src_iz=(0,) * 5, src_ix=(0, 17, 34, 52, 69), rec_iz=(0,) * 70,
                       rec_ix=tuple(range(70)), batch=4)
    c = api.coarse_problem(prob)
    assert (c.nz, c.nx, c.nb, c.nt, c.dx, c.dz, c.dt) == (35, 35, 20, 500, 20.0, 20.0, 2e-3)
    assert list(c.src_ix) == [0, 8, 17, 26, 34] and len(c.rec_ix) == 35
    assert list(c.rec_ix) == list(range(35))
    api.fwi_plan_create(c, api.W2Params())     # a valid plan (CFL bound unchanged)


def test_conv_wait_check_needs_a_status_word(api):
    p = ctypes.c_void_p(4096)
    assert api._lib.fwi_conv3x3_bf16_wait_check(1, 4, 4, 64, 64, p, p, p, 0, None, None) == 1
    assert "status" in api.fwi_last_error()


def test_forward_wait_check_needs_a_cluster_plan(api):
    prob = api.Problem(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3,
                       src_iz=(0,) * 5, src_ix=(0, 17, 34, 52, 69), rec_iz=(0,) * 70,
                       rec_ix=tuple(range(70)), batch=2)
    h = api.fwi_plan_create(prob, api.W2Params())     # resident kernels
    p = ctypes.c_void_p(4096)
    assert api._lib.fwi_forward_wait_check(h.raw, p, p, p, p, None) == api.FWI_ERR_UNSUPPORTED
    assert api._lib.fwi_forward_wait_check(None, p, p, p, p, None) == api.FWI_ERR_INVALID_ARG
