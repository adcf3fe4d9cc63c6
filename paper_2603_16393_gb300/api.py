"""Thin Python binding of libfwi.so (C ABI in include/fwi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and the current CUDA stream.  The
module refuses to import when libfwi.so is missing: there is no fallback.

Functions named ``fwi_*`` take the same arguments as the C entry points, with
torch tensors in place of device pointers.  :class:`Plan` bundles a plan with
the buffers it needs and offers the whole gradient in one call.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfwi.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

# status codes (fwi_status)
FWI_OK = 0
FWI_ERR_INVALID_ARG = 1
FWI_ERR_UNSTABLE_CFL = 2
FWI_ERR_UNSUPPORTED = 3
FWI_ERR_CUDA = 4
FWI_ERR_DEVICE_TIMEOUT = 5
FWI_ERR_OOM = 6
KERNELS_AUTO, KERNELS_RESIDENT, KERNELS_TILED, KERNELS_CLUSTER, KERNELS_CPML = 0, 1, 2, 3, 4
ABSORBER_SPONGE, ABSORBER_CPML = 0, 1
(SHAPE_DEFAULT, SHAPE_RESIDENT_PAIRS, SHAPE_RESIDENT_COLUMNS, SHAPE_CLUSTER_RS13,
 SHAPE_CLUSTER_RS19, SHAPE_TILED_ROWS8, SHAPE_TILED_ROWS4, SHAPE_CLUSTER_PAIRS,
 SHAPE_TILED_QUADS) = range(9)
SIGMA_POSTERIOR, SIGMA_BETA = 0, 1
FWI_MAX_SHOTS = 256
FWI_MAX_RECEIVERS = 1024
FWI_QUEUE_MAX_PLANS = 4

_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


class _Problem(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("dz", ctypes.c_double),
                ("dx", ctypes.c_double), ("nb", ctypes.c_int), ("top_bc", ctypes.c_int),
                ("nt", ctypes.c_int), ("dt", ctypes.c_double), ("ns", ctypes.c_int),
                ("nr", ctypes.c_int), ("src_iz", _ip), ("src_ix", _ip), ("rec_iz", _ip),
                ("rec_ix", _ip), ("f_peak", ctypes.c_double), ("t0", ctypes.c_double),
                ("v_ref", ctypes.c_double), ("refl_R", ctypes.c_double),
                ("v_max", ctypes.c_double), ("batch", ctypes.c_int),
                ("checkpoint_every", ctypes.c_int), ("space_order", ctypes.c_int),
                ("kernels", ctypes.c_int), ("absorber", ctypes.c_int),
                ("shape", ctypes.c_int)]


class _W2(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("cshift_factor", ctypes.c_double),
                ("eps_density", ctypes.c_double), ("n_xi", ctypes.c_int),
                ("squared", ctypes.c_int)]


class _Guide(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("rho0", "c", "tau", "gamma", "eps", "kappa_min", "kappa_max", "unit")]


class _DdpmStep(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("abar", "c_v", "c_0", "sigma")]


class _Space(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("shift", "unit", "v_lo", "v_hi")]


_S = ctypes.c_int
_lib.fwi_plan_create.restype = _S
_lib.fwi_plan_create.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_W2), ctypes.POINTER(_vp)]
_lib.fwi_plan_destroy.restype = None
_lib.fwi_plan_destroy.argtypes = [_vp]
_lib.fwi_plan_sizes.restype = _S
_lib.fwi_plan_sizes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
_lib.fwi_plan_padded.restype = _S
_lib.fwi_plan_padded.argtypes = [_vp, _ip, _ip]
_lib.fwi_plan_kernels.restype = _S
_lib.fwi_plan_kernels.argtypes = [_vp, _ip]
_lib.fwi_forward.restype = _S
_lib.fwi_forward.argtypes = [_vp] * 6
_lib.fwi_w2_prepare.restype = _S
_lib.fwi_w2_prepare.argtypes = [_vp] * 4
_lib.fwi_w2_misfit.restype = _S
_lib.fwi_w2_misfit.argtypes = [_vp] * 8
_lib.fwi_adjoint_grad.restype = _S
_lib.fwi_adjoint_grad.argtypes = [_vp] * 7
_lib.fwi_guided_step.restype = _S
_lib.fwi_guided_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(_Guide)] + [_vp] * 7
_lib.fwi_w2_misfit_static.restype = _S
_lib.fwi_w2_misfit_static.argtypes = [_vp] * 7
_lib.fwi_l2_misfit.restype = _S
_lib.fwi_l2_misfit.argtypes = [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]
_lib.fwi_tv_grad.restype = _S
_lib.fwi_tv_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, _vp, _vp, _vp, _vp, _vp]
_lib.fwi_image_metrics.restype = _S
_lib.fwi_image_metrics.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   _vp, _vp, _vp, _vp]
_lib.fwi_autotune_scratch_bytes.restype = _S
_lib.fwi_autotune_scratch_bytes.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
_lib.fwi_autotune_kernels.restype = _S
_lib.fwi_autotune_kernels.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_int), _vp]
_lib.fwi_queue_forward.restype = _S
_lib.fwi_queue_forward.argtypes = [ctypes.POINTER(_vp), ctypes.c_int] + [ctypes.POINTER(_vp)] * 4 + \
    [_vp, _vp]
_lib.fwi_queue_adjoint.restype = _S
_lib.fwi_queue_adjoint.argtypes = [ctypes.POINTER(_vp), ctypes.c_int] + [ctypes.POINTER(_vp)] * 5 + \
    [_vp, _vp]
_lib.fwi_group_create.restype = _S
_lib.fwi_group_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp)]
_lib.fwi_group_destroy.restype = None
_lib.fwi_group_destroy.argtypes = [_vp]
_lib.fwi_group_gradient.restype = _S
_lib.fwi_group_gradient.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 8 + [_vp]
_lib.fwi_ddpm_coefficients.restype = _S
_lib.fwi_ddpm_coefficients.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(_DdpmStep)]
_lib.fwi_ddpm_proposal.restype = _S
_lib.fwi_ddpm_proposal.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_DdpmStep),
                                   ctypes.POINTER(_Space)] + [_vp] * 9
_lib.fwi_ddpm_guidance.restype = _S
_lib.fwi_ddpm_guidance.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_DdpmStep),
                                   ctypes.POINTER(_Space)] + [_vp] * 7
_lib.fwi_conv3x3_bf16.restype = _S
_lib.fwi_conv3x3_bf16.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp, ctypes.c_int, _vp,
                                                       ctypes.c_int, _vp, _vp]
_lib.fwi_conv3x3_bf16_silu.restype = _S
_lib.fwi_conv3x3_bf16_silu.argtypes = [ctypes.c_int] * 5 + [_vp] * 7
_lib.fwi_conv3x3_bf16_silu_grad.restype = _S
_lib.fwi_conv3x3_bf16_silu_grad.argtypes = [ctypes.c_int] * 5 + [_vp] * 6
_lib.fwi_restrict2.restype = _S
_lib.fwi_restrict2.argtypes = [ctypes.c_int] * 3 + [_vp] * 3
_lib.fwi_restrict2_transpose.restype = _S
_lib.fwi_restrict2_transpose.argtypes = [ctypes.c_int] * 3 + [_vp] * 3
_lib.fwi_decimate2.restype = _S
_lib.fwi_decimate2.argtypes = [ctypes.c_int] * 4 + [_vp] * 3
_lib.fwi_coarse_problem.restype = _S
_lib.fwi_coarse_problem.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Problem)] + [_ip] * 4
_lib.fwi_pack_channel0.restype = _S
_lib.fwi_pack_channel0.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_float, _vp, _vp, _vp]
_lib.fwi_unpack_channel0.restype = _S
_lib.fwi_unpack_channel0.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_float, _vp, _vp,
                                     _vp]
_lib.fwi_silu_bf16.restype = _S
_lib.fwi_silu_bf16.argtypes = [ctypes.c_longlong, _vp, _vp, _vp]
_lib.fwi_silu_grad_bf16.restype = _S
_lib.fwi_silu_grad_bf16.argtypes = [ctypes.c_longlong, _vp, _vp, _vp, _vp]
_lib.fwi_conv3x3_bf16_wait_check.restype = _S
_lib.fwi_conv3x3_bf16_wait_check.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp, ctypes.c_int,
                                                                  _vp, _vp]
_lib.fwi_forward_wait_check.restype = _S
_lib.fwi_forward_wait_check.argtypes = [_vp] * 6
_lib.fwi_dsm_noisy.restype = _S
_lib.fwi_dsm_noisy.argtypes = [ctypes.c_longlong, ctypes.c_double, _vp, _vp, _vp, _vp]
_lib.fwi_dsm_loss.restype = _S
_lib.fwi_dsm_loss.argtypes = [ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp]
_lib.fwi_conv3x3_wgrad.restype = _S
_lib.fwi_conv3x3_wgrad.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp, _vp, ctypes.c_longlong,
                                                         _vp]
_lib.fwi_conv3x3_wgrad_tc.restype = _S
_lib.fwi_conv3x3_wgrad_tc.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp, _vp, ctypes.c_longlong,
                                                            _vp, ctypes.c_longlong, _vp, _vp]
_lib.fwi_conv3x3_wgrad_tc_wait_check.restype = _S
_lib.fwi_conv3x3_wgrad_tc_wait_check.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp, _vp,
                                                                       ctypes.c_longlong, _vp,
                                                                       _vp]
_lib.fwi_conv3x3_wgrad_tc_stage_bytes.restype = ctypes.c_longlong
_lib.fwi_conv3x3_wgrad_tc_stage_bytes.argtypes = [ctypes.c_int] * 5
_lib.fwi_conv3x3_wgrad_tc_splits.restype = ctypes.c_int
_lib.fwi_conv3x3_wgrad_tc_splits.argtypes = [ctypes.c_int] * 5 + [ctypes.c_longlong]
_lib.fwi_conv3x3_wgrad_splits.restype = ctypes.c_int
_lib.fwi_conv3x3_wgrad_splits.argtypes = [ctypes.c_int] * 5 + [ctypes.c_longlong]
_lib.fwi_pool2_bf16.restype = _S
_lib.fwi_pool2_bf16.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp]
_lib.fwi_up2_bf16.restype = _S
_lib.fwi_up2_bf16.argtypes = [ctypes.c_int] * 5 + [_vp, _vp, _vp]
_lib.fwi_add_bf16.restype = _S
_lib.fwi_add_bf16.argtypes = [ctypes.c_longlong, _vp, _vp, _vp, _vp]
_i, _f = ctypes.c_int, ctypes.c_float
_lib.fwi_ddpm_table.restype = _S
_lib.fwi_ddpm_table.argtypes = [ctypes.POINTER(ctypes.c_double), _i, _i, ctypes.c_void_p, _vp]
_lib.fwi_ddpm_proposal_at.restype = _S
_lib.fwi_ddpm_proposal_at.argtypes = [_i, _i, _vp, _vp, _i] + [_vp] * 5 + [ctypes.c_longlong] + \
    [_vp] * 4
_lib.fwi_ddpm_guidance_at.restype = _S
_lib.fwi_ddpm_guidance_at.argtypes = [_i, _i, _vp, _vp, _i] + [_vp] * 7
_lib.fwi_ddpm_step_down.restype = _S
_lib.fwi_ddpm_step_down.argtypes = [_vp, _vp]
_lib.fwi_sur_pack.restype = _S
_lib.fwi_sur_pack.argtypes = [_i] * 5 + [_f, _f] + [_vp] * 4
_lib.fwi_sur_unpack_grad.restype = _S
_lib.fwi_sur_unpack_grad.argtypes = [_i] * 5 + [_f] + [_vp] * 3
_lib.fwi_sur_traces.restype = _S
_lib.fwi_sur_traces.argtypes = [_i] * 7 + [_f] + [_vp] * 4
_lib.fwi_sur_output_grad.restype = _S
_lib.fwi_sur_output_grad.argtypes = [_i] * 7 + [_f, _f] + [_vp] * 5
_lib.fwi_sur_target.restype = _S
_lib.fwi_sur_target.argtypes = [_i] * 7 + [_f] + [_vp] * 4
_lib.fwi_sur_loss.restype = _S
_lib.fwi_sur_loss.argtypes = [ctypes.c_longlong] + [_vp] * 5 + [ctypes.c_longlong, _vp]
_lib.fwi_pool_h_bf16.restype = _S
_lib.fwi_pool_h_bf16.argtypes = [_i] * 5 + [_vp] * 3
_lib.fwi_up_h_bf16.restype = _S
_lib.fwi_up_h_bf16.argtypes = [_i] * 5 + [_vp] * 3
_lib.fwi_sur_weights_prep.restype = _S
_lib.fwi_sur_weights_prep.argtypes = [_i, _i] + [_vp] * 4
_lib.fwi_sur_wgrad_centre.restype = _S
_lib.fwi_sur_wgrad_centre.argtypes = [_i, _i] + [_vp] * 3
_lib.fwi_lowrank_score_at.restype = _S
_lib.fwi_lowrank_score_at.argtypes = [_i, _i, _i, _vp, _vp, ctypes.c_double] + [_vp] * 4 + \
    [_i] + [_vp] * 3
_lib.fwi_rel_error.restype = _S
_lib.fwi_rel_error.argtypes = [_i, ctypes.c_longlong] + [_vp] * 4
_lib.fwi_channel_sum.restype = _S
_lib.fwi_channel_sum.argtypes = [ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp, ctypes.c_longlong,
                                 _vp]
_lib.fwi_adam_step.restype = _S
_lib.fwi_adam_step.argtypes = [ctypes.c_longlong] + [ctypes.c_double] * 4 + [ctypes.c_int] + \
    [_vp] * 5
_lib.fwi_conv3x3_weights_prep.restype = _S
_lib.fwi_conv3x3_weights_prep.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.fwi_time_bias.restype = _S
_lib.fwi_time_bias.argtypes = [ctypes.c_int] * 3 + [_vp] * 5
_lib.fwi_time_bias_grad.restype = _S
_lib.fwi_time_bias_grad.argtypes = [ctypes.c_int] * 2 + [_vp] * 4
_lib.fwi_check.restype = _S
_lib.fwi_check.argtypes = [_vp, _vp, _vp]
_lib.fwi_last_error.restype = ctypes.c_char_p
_lib.fwi_last_error.argtypes = []
_lib.fwi_version.restype = ctypes.c_int
_lib.fwi_version.argtypes = []


class FwiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fwi status {code}: {msg}")
        self.code = code


def _check(code: int):
    if code != FWI_OK:
        raise FwiError(code, _lib.fwi_last_error().decode())


def fwi_version() -> int:
    return _lib.fwi_version()


def fwi_last_error() -> str:
    return _lib.fwi_last_error().decode()


# ----------------------------------------------------------------- parameter mirrors

@dataclasses.dataclass
class Problem:
    """Mirror of ``fwi_problem`` (see include/fwi.h for every field)."""
    nz: int
    nx: int
    nb: int
    nt: int
    dz: float
    dx: float
    dt: float
    src_iz: Sequence[int]
    src_ix: Sequence[int]
    rec_iz: Sequence[int]
    rec_ix: Sequence[int]
    f_peak: float = 15.0
    t0: float = 0.0
    v_ref: float = 4500.0
    refl_R: float = 1e-3
    v_max: float = 4500.0
    batch: int = 1
    top_bc: int = 0
    checkpoint_every: int = 0     # 0: keep the whole record; K: checkpoint every K steps
    space_order: int = 4          # 4 or 8 (8: the paper solver's stencil, tiled kernels)
    kernels: int = 0              # propagator family: KERNELS_AUTO / _RESIDENT / _TILED / _CLUSTER / _CPML
    absorber: int = 0             # ABSORBER_SPONGE (damping layer) or ABSORBER_CPML
    shape: int = 0                # thread shape inside the family (SHAPE_*; 0: default)

    @property
    def ns(self):
        return len(self.src_ix)

    @property
    def nr(self):
        return len(self.rec_ix)

    @property
    def NZ(self):
        return self.nz + self.nb

    @property
    def NX(self):
        return self.nx + 2 * self.nb


@dataclasses.dataclass
class W2Params:
    """Mirror of ``fwi_w2_params``; defaults are the paper's (Sec. 6.2, 6.3)."""
    k: float = 100.0
    cshift_factor: float = 1.1
    eps_density: float = 1e-9
    n_xi: int = 1000
    squared: bool = False   # True: sum W2^2 / sum |Q_obs|^2 (W2+TV baseline; use k = 0)


@dataclasses.dataclass
class GuideParams:
    """Mirror of ``fwi_guide_params``; c, tau, eps default to Sec. 6.3."""
    rho0: float = 1.0
    c: float = 0.1
    tau: float = 0.0
    gamma: float = 0.5
    eps: float = 1e-4
    kappa_min: float = 0.0
    kappa_max: float = 0.0
    unit: float = 1.0        # one normalised-space unit in the units of the arrays

    def _c(self):
        return _Guide(*(float(getattr(self, f)) for f, _ in _Guide._fields_))


@dataclasses.dataclass(frozen=True)
class DdpmStep:
    """Coefficients of one reverse step (fwi_ddpm_step): abar_i and
    v' = c_v v_i + c_0 v0hat + sigma z."""
    abar: float
    c_v: float
    c_0: float
    sigma: float

    def _c(self):
        return _DdpmStep(self.abar, self.c_v, self.c_0, self.sigma)


@dataclasses.dataclass(frozen=True)
class DiffusionSpace:
    """Normalised diffusion space x = (v - shift) / unit and the clamp of the
    physics model (fwi_diffusion_space)."""
    shift: float = 3000.0
    unit: float = 1500.0
    v_lo: float = 1500.0
    v_hi: float = 4500.0

    def _c(self):
        return _Space(self.shift, self.unit, self.v_lo, self.v_hi)


# ----------------------------------------------------------------- marshalling helpers

def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, shape, name):
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class _Handle:
    def __init__(self, raw):
        self.raw = raw

    def __del__(self):
        if self.raw:
            _lib.fwi_plan_destroy(self.raw)
            self.raw = None


def _c_problem(prob: Problem, w2: W2Params):
    """C structs of a problem and its W2 parameters (the index arrays are
    returned too: they must outlive the call)."""
    if len(prob.src_iz) != len(prob.src_ix) or len(prob.rec_iz) != len(prob.rec_ix):
        raise ValueError("source/receiver index lists differ in length")
    arrays = [(ctypes.c_int * len(a))(*[int(x) for x in a])
              for a in (prob.src_iz, prob.src_ix, prob.rec_iz, prob.rec_ix)]
    cp = _Problem(prob.nz, prob.nx, prob.dz, prob.dx, prob.nb, prob.top_bc, prob.nt, prob.dt,
                  len(prob.src_ix), len(prob.rec_ix),
                  *[ctypes.cast(a, _ip) for a in arrays],
                  prob.f_peak, prob.t0, prob.v_ref, prob.refl_R, prob.v_max, prob.batch,
                  prob.checkpoint_every, prob.space_order, prob.kernels, prob.absorber,
                  prob.shape)
    cw = _W2(w2.k, w2.cshift_factor, w2.eps_density, w2.n_xi, int(w2.squared))
    return cp, cw, arrays


def fwi_plan_create(prob: Problem, w2: W2Params) -> _Handle:
    cp, cw, _arrays = _c_problem(prob, w2)
    out = _vp()
    _check(_lib.fwi_plan_create(ctypes.byref(cp), ctypes.byref(cw), ctypes.byref(out)))
    return _Handle(out)


def fwi_autotune_scratch_bytes(prob: Problem, w2: W2Params, trial_steps: int) -> int:
    cp, cw, _arrays = _c_problem(prob, w2)
    n = ctypes.c_size_t()
    _check(_lib.fwi_autotune_scratch_bytes(ctypes.byref(cp), ctypes.byref(cw), int(trial_steps),
                                           ctypes.byref(n)))
    return n.value


def fwi_autotune_kernels(prob: Problem, w2: W2Params, v, trial_steps: int, scratch, stream=None):
    """(fastest family, its fastest shape, predicted ms of a pass at nt for
    [resident, tiled, cluster, CPML] each at its fastest shape, those shapes)
    -- -1 where a family cannot run the problem."""
    cp, cw, _arrays = _c_problem(prob, w2)
    fam, shape = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 4)()
    shapes = (ctypes.c_int * 4)()
    _check(_lib.fwi_autotune_kernels(ctypes.byref(cp), ctypes.byref(cw), _ptr(v), int(trial_steps),
                                     _ptr(scratch), scratch.numel() * scratch.element_size(),
                                     ctypes.byref(fam), ctypes.byref(shape), ms, shapes,
                                     _stream(stream)))
    return fam.value, shape.value, [float(t) for t in ms], [int(x) for x in shapes]


def fwi_plan_sizes(plan: _Handle):
    ws, ctx, snap = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.fwi_plan_sizes(plan.raw, ctypes.byref(ws), ctypes.byref(ctx), ctypes.byref(snap)))
    return ws.value, ctx.value, snap.value


def fwi_plan_kernels(plan: _Handle) -> int:
    fam = ctypes.c_int()
    _check(_lib.fwi_plan_kernels(plan.raw, ctypes.byref(fam)))
    return fam.value


def fwi_forward(plan, v, d_syn, snapshots, workspace, stream=None):
    _check(_lib.fwi_forward(plan.raw, _ptr(v), _ptr(d_syn), _ptr(snapshots), _ptr(workspace),
                            _stream(stream)))


def fwi_forward_wait_check(plan, v, d_syn, snapshots, workspace, stream=None):
    """The cluster kernels' bounded-wait self-check (see include/fwi.h)."""
    _check(_lib.fwi_forward_wait_check(plan.raw, _ptr(v), _ptr(d_syn), _ptr(snapshots),
                                       _ptr(workspace), _stream(stream)))


def fwi_w2_prepare(plan, d_obs, obs_ctx, stream=None):
    _check(_lib.fwi_w2_prepare(plan.raw, _ptr(d_obs), _ptr(obs_ctx), _stream(stream)))


def fwi_w2_misfit(plan, obs_ctx, d_syn, J, w2, adj_src, workspace, stream=None):
    _check(_lib.fwi_w2_misfit(plan.raw, _ptr(obs_ctx), _ptr(d_syn), _ptr(J), _ptr(w2),
                              _ptr(adj_src), _ptr(workspace), _stream(stream)))


def fwi_w2_misfit_static(plan, obs_ctx, d_syn, J, w2, adj_src, stream=None):
    _check(_lib.fwi_w2_misfit_static(plan.raw, _ptr(obs_ctx), _ptr(d_syn), _ptr(J), _ptr(w2),
                                     _ptr(adj_src), _stream(stream)))


FWI_STATIC_MAX_TRACES = 65536


def fwi_adjoint_grad(plan, v, adj_src, snapshots, grad, workspace, stream=None):
    _check(_lib.fwi_adjoint_grad(plan.raw, _ptr(v), _ptr(adj_src), _ptr(snapshots), _ptr(grad),
                                 _ptr(workspace), _stream(stream)))


def fwi_guided_step(batch, nz, nx, params: GuideParams, v_prime, v0hat, g, h, v_out, rho_out,
                    stream=None):
    gp = params._c()
    _check(_lib.fwi_guided_step(batch, nz, nx, ctypes.byref(gp), _ptr(v_prime), _ptr(v0hat),
                                _ptr(g), _ptr(h), _ptr(v_out), _ptr(rho_out), _stream(stream)))


def fwi_l2_misfit(plan, d_obs, d_syn, sigma, J, adj_src, stream=None):
    _check(_lib.fwi_l2_misfit(plan.raw, _ptr(d_obs), _ptr(d_syn), ctypes.c_double(sigma),
                              _ptr(J), _ptr(adj_src), _stream(stream)))


def fwi_tv_grad(batch, nz, nx, alpha, unit, v, g, h, tv, stream=None):
    _check(_lib.fwi_tv_grad(batch, nz, nx, ctypes.c_double(alpha), ctypes.c_double(unit),
                            _ptr(v), _ptr(g), _ptr(h), _ptr(tv), _stream(stream)))


def fwi_image_metrics(batch, nz, nx, data_range, v_true, v_rec, out, stream=None):
    _check(_lib.fwi_image_metrics(batch, nz, nx, ctypes.c_double(data_range), _ptr(v_true),
                                  _ptr(v_rec), _ptr(out), _stream(stream)))


def fwi_ddpm_coefficients(betas: Sequence[float], i: int,
                          sigma_mode: int = SIGMA_POSTERIOR) -> DdpmStep:
    b = (ctypes.c_double * len(betas))(*[float(x) for x in betas])
    out = _DdpmStep()
    _check(_lib.fwi_ddpm_coefficients(b, len(betas), int(i), int(sigma_mode), ctypes.byref(out)))
    return DdpmStep(out.abar, out.c_v, out.c_0, out.sigma)


def fwi_ddpm_proposal(batch, ncell, step: DdpmStep, space: DiffusionSpace, v_i, score, mu, tau2,
                      z, v0hat, v_prime, v_phys, stream=None):
    st, sp = step._c(), space._c()
    _check(_lib.fwi_ddpm_proposal(batch, ncell, ctypes.byref(st), ctypes.byref(sp), _ptr(v_i),
                                  _ptr(score), _ptr(mu), _ptr(tau2), _ptr(z), _ptr(v0hat),
                                  _ptr(v_prime), _ptr(v_phys), _stream(stream)))


def fwi_ddpm_guidance(batch, ncell, step: DdpmStep, space: DiffusionSpace, v0hat, g_phys, vjp,
                      tau2, g, h, stream=None):
    st, sp = step._c(), space._c()
    _check(_lib.fwi_ddpm_guidance(batch, ncell, ctypes.byref(st), ctypes.byref(sp), _ptr(v0hat),
                                  _ptr(g_phys), _ptr(vjp), _ptr(tau2), _ptr(g), _ptr(h),
                                  _stream(stream)))



DDPM_RECORD_FLOATS = 12


def ddpm_table(betas, sigma_mode=0, space=None, device=None) -> torch.Tensor:
    """The device table of every step's coefficients for the graph-replayed
    reverse step (fwi_ddpm_table; records of DDPM_RECORD_FLOATS floats, record
    i for step i)."""
    space = space if space is not None else DiffusionSpace()
    b = (ctypes.c_double * len(betas))(*[float(x) for x in betas])
    host = torch.zeros((len(betas) + 1) * DDPM_RECORD_FLOATS, dtype=torch.float32)
    sp = _Space(space.shift, space.unit, space.v_lo, space.v_hi)
    _check(_lib.fwi_ddpm_table(b, len(betas), int(sigma_mode), ctypes.byref(sp),
                               ctypes.c_void_p(host.data_ptr())))
    return host.to(device or torch.device("cuda"))


def fwi_ddpm_proposal_at(batch, ncell, table, step, n_steps, v_i, score, mu, tau2, z, z_stride,
                         v0hat, v_prime, v_phys, stream=None):
    """fwi_ddpm_proposal at the device step index *step (int32 [1]); z is the
    first of the per-step draws, step i reading z + i z_stride."""
    if step.dtype != torch.int32 or step.numel() != 1 or not step.is_cuda:
        raise ValueError("step must be one int32 on the device")
    if z.numel() < (n_steps + 1) * z_stride:
        raise ValueError("z holds fewer than (n_steps + 1) z_stride draws")
    _check(_lib.fwi_ddpm_proposal_at(batch, ncell, _ptr(table), _ptr(step), n_steps, _ptr(v_i),
                                     _ptr(score), _ptr(mu), _ptr(tau2), _ptr(z), int(z_stride),
                                     _ptr(v0hat), _ptr(v_prime), _ptr(v_phys), _stream(stream)))


def fwi_ddpm_guidance_at(batch, ncell, table, step, n_steps, v0hat, g_phys, vjp, tau2, g, h,
                         stream=None):
    if step.dtype != torch.int32 or step.numel() != 1 or not step.is_cuda:
        raise ValueError("step must be one int32 on the device")
    _check(_lib.fwi_ddpm_guidance_at(batch, ncell, _ptr(table), _ptr(step), n_steps, _ptr(v0hat),
                                     _ptr(g_phys), _ptr(vjp), _ptr(tau2), _ptr(g), _ptr(h),
                                     _stream(stream)))


def fwi_lowrank_score_at(batch, ncell, U, lam, s2, x, mu, table, step, n_steps, work, out,
                         stream=None):
    """Score of the low-rank Gaussian prior N(mu, U^T diag(lam) U + s2 I) at
    step *step: out = -C^-1 (x - sqrt(abar) mu), or with mu None -C^-1 x (the
    score's vector-Jacobian product applied to x).  U [k][ncell] (orthonormal
    rows), lam [k], x and out [batch][ncell], work [batch][k]; fp32 device."""
    k = 0 if U is None else U.shape[0]
    if step.dtype != torch.int32 or step.numel() != 1 or not step.is_cuda:
        raise ValueError("step must be one int32 on the device")
    if k:
        _f32(U, (k, ncell), "U")
        _f32(lam, (k,), "lam")
        if work is None or work.numel() < batch * k:
            raise ValueError("work must hold batch x k floats")
    _check(_lib.fwi_lowrank_score_at(batch, ncell, k, _ptr(U), _ptr(lam), float(s2), _ptr(x),
                                     _ptr(mu), _ptr(table), _ptr(step), n_steps, _ptr(work),
                                     _ptr(out), _stream(stream)))


def fwi_ddpm_step_down(step, stream=None):
    _check(_lib.fwi_ddpm_step_down(_ptr(step), _stream(stream)))


def fwi_conv3x3_bf16(x, wt, bias, act, y, status=None, stream=None):
    """3x3 convolution on the tensor cores: x [n][h][w][cin] bf16, wt
    [cout][3][3][cin] bf16, bias [cout] fp32 or None, y [n][h][w][cout] fp32 or
    bf16 (all contiguous CUDA tensors); act 0 identity, 1 SiLU."""
    n, h, w, cin = x.shape
    cout = wt.shape[0]
    if x.dtype != torch.bfloat16 or wt.dtype != torch.bfloat16:
        raise TypeError("x and wt must be bfloat16")
    if tuple(wt.shape) != (cout, 3, 3, cin):
        raise ValueError(f"wt must have shape {(cout, 3, 3, cin)}, got {tuple(wt.shape)}")
    if tuple(y.shape) != (n, h, w, cout) or y.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("y must be [n][h][w][cout] float32 or bfloat16")
    if bias is not None:
        _f32(bias, (cout,), "bias")
    _check(_lib.fwi_conv3x3_bf16(n, h, w, cin, cout, _ptr(x), _ptr(wt), _ptr(bias), int(act),
                                 _ptr(y), int(y.dtype == torch.bfloat16), _ptr(status),
                                 _stream(stream)))


def fwi_conv3x3_bf16_silu(x, wt, bias, p, a, status=None, stream=None):
    """The convolution writing both bf16 outputs of a layer: p the
    pre-activation and a = SiLU(p), bit for bit fwi_conv3x3_bf16 (act 0, bf16
    out) followed by fwi_silu_bf16."""
    n, h, w, cin = x.shape
    cout = wt.shape[0]
    if x.dtype != torch.bfloat16 or wt.dtype != torch.bfloat16:
        raise TypeError("x and wt must be bfloat16")
    if tuple(wt.shape) != (cout, 3, 3, cin):
        raise ValueError(f"wt must have shape {(cout, 3, 3, cin)}, got {tuple(wt.shape)}")
    for t, nm in ((p, "p"), (a, "a")):
        if tuple(t.shape) != (n, h, w, cout) or t.dtype != torch.bfloat16:
            raise ValueError(f"{nm} must be [n][h][w][cout] bfloat16")
    if bias is not None:
        _f32(bias, (cout,), "bias")
    _check(_lib.fwi_conv3x3_bf16_silu(n, h, w, cin, cout, _ptr(x), _ptr(wt), _ptr(bias), _ptr(p),
                                      _ptr(a), _ptr(status), _stream(stream)))


def fwi_conv3x3_bf16_silu_grad(x, wt, p, dp, status=None, stream=None):
    """The convolution (no bias) carrying a gradient x back through a layer,
    times the SiLU derivative at the pre-activation p of the layer below: bit
    for bit fwi_conv3x3_bf16 (act 0, bf16 out) followed by
    fwi_silu_grad_bf16."""
    n, h, w, cin = x.shape
    cout = wt.shape[0]
    if x.dtype != torch.bfloat16 or wt.dtype != torch.bfloat16:
        raise TypeError("x and wt must be bfloat16")
    if tuple(wt.shape) != (cout, 3, 3, cin):
        raise ValueError(f"wt must have shape {(cout, 3, 3, cin)}, got {tuple(wt.shape)}")
    for t, nm in ((p, "p"), (dp, "dp")):
        if tuple(t.shape) != (n, h, w, cout) or t.dtype != torch.bfloat16:
            raise ValueError(f"{nm} must be [n][h][w][cout] bfloat16")
    _check(_lib.fwi_conv3x3_bf16_silu_grad(n, h, w, cin, cout, _ptr(x), _ptr(wt), _ptr(p),
                                           _ptr(dp), _ptr(status), _stream(stream)))


def fwi_conv3x3_bf16_wait_check(x, wt, y, status, stream=None):
    """The convolution's bounded-wait self-check (see include/fwi.h): sets
    status[0] to FWI_ERR_DEVICE_TIMEOUT and leaves y unwritten."""
    n, h, w, cin = x.shape
    _check(_lib.fwi_conv3x3_bf16_wait_check(n, h, w, cin, wt.shape[0], _ptr(x), _ptr(wt),
                                            _ptr(y), int(y.dtype == torch.bfloat16),
                                            _ptr(status), _stream(stream)))


def conv3x3(x, wt, bias=None, act=0, out_dtype=torch.float32, status=None, stream=None):
    """Allocating form of fwi_conv3x3_bf16; returns y."""
    n, h, w, _ = x.shape
    y = torch.empty((n, h, w, wt.shape[0]), dtype=out_dtype, device=x.device)
    fwi_conv3x3_bf16(x, wt, bias, act, y, status, stream)
    return y


def fwi_restrict2(v, vc=None, stream=None):
    """R of the low-fidelity surrogate: 2 x 2 block means of [B][nz][nx] float32."""
    B, nz, nx = v.shape
    shape = (B, (nz + 1) // 2, (nx + 1) // 2)
    _f32(v, (B, nz, nx), "v")
    if vc is None:
        vc = torch.empty(shape, dtype=torch.float32, device=v.device)
    _f32(vc, shape, "vc")
    _check(_lib.fwi_restrict2(B, nz, nx, _ptr(v), _ptr(vc), _stream(stream)))
    return vc


def fwi_restrict2_transpose(gc, nz, nx, g=None, stream=None):
    """R^T: the fine-grid gradient of a function of R v from its coarse gradient."""
    B = gc.shape[0]
    _f32(gc, (B, (nz + 1) // 2, (nx + 1) // 2), "gc")
    if g is None:
        g = torch.empty((B, nz, nx), dtype=torch.float32, device=gc.device)
    _f32(g, (B, nz, nx), "g")
    _check(_lib.fwi_restrict2_transpose(B, nz, nx, _ptr(gc), _ptr(g), _stream(stream)))
    return g


def fwi_decimate2(d, dc=None, stream=None):
    """The coarse problem's observations: even receivers, samples 2m + 1."""
    B, ns, nr, nt = d.shape
    shape = (B, ns, (nr + 1) // 2, nt // 2)
    _f32(d, (B, ns, nr, nt), "d")
    if dc is None:
        dc = torch.empty(shape, dtype=torch.float32, device=d.device)
    _f32(dc, shape, "dc")
    _check(_lib.fwi_decimate2(B, ns, nr, nt, _ptr(d), _ptr(dc), _stream(stream)))
    return dc


def coarse_problem(prob: Problem) -> Problem:
    """The low-fidelity twin of a problem (fwi_restrict2 and friends), as the
    library's fwi_coarse_problem derives it: grid, spacing and time step
    doubled, nb rounded up, nt / 2 steps, sources at the coarse cells index / 2,
    the even receivers likewise."""
    cp, _cw, _arrays = _c_problem(prob, W2Params())
    out = _Problem()
    idx = [(ctypes.c_int * max(1, n))() for n in
           (prob.ns, prob.ns, (prob.nr + 1) // 2, (prob.nr + 1) // 2)]
    _check(_lib.fwi_coarse_problem(ctypes.byref(cp), ctypes.byref(out),
                                   *[ctypes.cast(a, _ip) for a in idx]))
    nrc = out.nr
    return dataclasses.replace(
        prob, nz=out.nz, nx=out.nx, nb=out.nb, nt=out.nt, dz=out.dz, dx=out.dx, dt=out.dt,
        src_iz=list(idx[0][:prob.ns]), src_ix=list(idx[1][:prob.ns]),
        rec_iz=list(idx[2][:nrc]), rec_ix=list(idx[3][:nrc]),
        checkpoint_every=out.checkpoint_every)


def fwi_pack_channel0(x, X, scale=1.0, stream=None):
    """X[..., 0] = bf16(scale x), other channels 0 (x [B][nz][nx] fp32, X [B][nz][nx][C] bf16)."""
    if X.dtype != torch.bfloat16 or tuple(X.shape[:-1]) != tuple(x.shape):
        raise ValueError("X must be bfloat16 of shape x.shape + (C,)")
    _f32(x, tuple(x.shape), "x")
    _check(_lib.fwi_pack_channel0(x.numel(), X.shape[-1], ctypes.c_float(scale), _ptr(x), _ptr(X),
                                  _stream(stream)))


def fwi_unpack_channel0(Y, y, scale=1.0, stream=None):
    """y = scale Y[..., 0] (Y [B][nz][nx][C] fp32, y [B][nz][nx] fp32)."""
    _f32(Y, tuple(Y.shape), "Y")
    _f32(y, tuple(Y.shape[:-1]), "y")
    _check(_lib.fwi_unpack_channel0(y.numel(), Y.shape[-1], ctypes.c_float(scale), _ptr(Y),
                                    _ptr(y), _stream(stream)))


def fwi_silu_bf16(P, A, stream=None):
    if P.dtype != torch.bfloat16 or A.dtype != torch.bfloat16 or P.shape != A.shape:
        raise ValueError("P and A must be bfloat16 tensors of one shape")
    _check(_lib.fwi_silu_bf16(P.numel(), _ptr(P), _ptr(A), _stream(stream)))


def fwi_silu_grad_bf16(dA, P, dP, stream=None):
    if not (dA.dtype == P.dtype == dP.dtype == torch.bfloat16) or not (dA.shape == P.shape == dP.shape):
        raise ValueError("dA, P and dP must be bfloat16 tensors of one shape")
    _check(_lib.fwi_silu_grad_bf16(P.numel(), _ptr(dA), _ptr(P), _ptr(dP), _stream(stream)))


def fwi_dsm_noisy(x0, z, abar, xt, stream=None):
    _check(_lib.fwi_dsm_noisy(x0.numel(), float(abar), _ptr(x0), _ptr(z), _ptr(xt),
                              _stream(stream)))


def _work(work):
    if work is None:
        return None, 0
    if work.dtype != torch.float32 or not work.is_contiguous():
        raise ValueError("work must be a contiguous float32 tensor")
    return _ptr(work), work.numel()


def fwi_dsm_loss(eps, z, loss, grad, work=None, stream=None):
    wp, wf = _work(work)
    _check(_lib.fwi_dsm_loss(eps.numel(), _ptr(eps), _ptr(z), _ptr(loss), _ptr(grad), wp, wf,
                             _stream(stream)))


WGRAD_MAX_SPLITS = 32   # partial tiles a work buffer of WGRAD_MAX_SPLITS 9 C^2 floats holds


def _wgrad_operands(X, dP, dW, work):
    n, h, w, cin = X.shape
    cout = dP.shape[-1]
    if X.dtype != torch.bfloat16 or dP.dtype != torch.bfloat16 or tuple(dP.shape[:3]) != (n, h, w):
        raise ValueError("X and dP must be bfloat16 [n][h][w][C] of one image shape")
    if not (X.is_contiguous() and dP.is_contiguous()):
        raise ValueError("X and dP must be contiguous")
    _f32(dW, (cout, 3, 3, cin), "dW")
    wp, wf = _work(work)
    return n, h, w, cin, cout, wp, wf


def fwi_conv3x3_wgrad(X, dP, dW, work=None, stream=None):
    """dW [cout][3][3][cin] float32 from X bf16 [n][h][w][cin] and dP bf16
    [n][h][w][cout] on the CUDA cores; ``work`` a float32 device buffer for the
    per-range partial sums (WGRAD_MAX_SPLITS 9 cin cout floats use every split
    the library wants; None: one range)."""
    n, h, w, cin, cout, wp, wf = _wgrad_operands(X, dP, dW, work)
    _check(_lib.fwi_conv3x3_wgrad(n, h, w, cin, cout, _ptr(X), _ptr(dP), _ptr(dW), wp, wf,
                                  _stream(stream)))


def fwi_conv3x3_wgrad_splits(n, h, w, cin, cout, work_floats):
    return _lib.fwi_conv3x3_wgrad_splits(n, h, w, cin, cout, work_floats)


def fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, cin, cout):
    return _lib.fwi_conv3x3_wgrad_tc_stage_bytes(n, h, w, cin, cout)


def fwi_conv3x3_wgrad_tc_splits(n, h, w, cin, cout, work_floats):
    return _lib.fwi_conv3x3_wgrad_tc_splits(n, h, w, cin, cout, work_floats)


def fwi_conv3x3_wgrad_tc(X, dP, dW, stage, work=None, status=None, stream=None):
    """The weight gradient on the tensor cores (cin, cout multiples of 64):
    ``stage`` a device buffer of at least fwi_conv3x3_wgrad_tc_stage_bytes
    bytes, ``work`` float32 for the partial tiles (None: one range)."""
    n, h, w, cin, cout, wp, wf = _wgrad_operands(X, dP, dW, work)
    if not stage.is_contiguous():
        raise ValueError("stage must be contiguous")
    _check(_lib.fwi_conv3x3_wgrad_tc(n, h, w, cin, cout, _ptr(X), _ptr(dP), _ptr(dW), _ptr(stage),
                                     stage.numel() * stage.element_size(), wp, wf, _ptr(status),
                                     _stream(stream)))


def fwi_conv3x3_wgrad_tc_wait_check(X, dP, dW, stage, status, stream=None):
    """The weight gradient's bounded-wait self-check: *status becomes
    FWI_ERR_DEVICE_TIMEOUT and the call returns normally."""
    n, h, w, cin, cout, _, _ = _wgrad_operands(X, dP, dW, None)
    _check(_lib.fwi_conv3x3_wgrad_tc_wait_check(n, h, w, cin, cout, _ptr(X), _ptr(dP), _ptr(dW),
                                                _ptr(stage), stage.numel() * stage.element_size(),
                                                _ptr(status), _stream(stream)))


def _bf16_nhwc(t, name):
    if t.dtype != torch.bfloat16 or t.dim() != 4 or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{name} must be a contiguous bfloat16 CUDA tensor [n][h][w][C]")


def fwi_pool2_bf16(x, y, mode=0, stream=None):
    """y [n][(h+1)/2][(w+1)/2][C] from x [n][h][w][C]: 2 x 2 block mean (mode 0)
    or sum (mode 1)."""
    _bf16_nhwc(x, "x")
    _bf16_nhwc(y, "y")
    n, h, w, c = x.shape
    if tuple(y.shape) != (n, (h + 1) // 2, (w + 1) // 2, c):
        raise ValueError("y must be [n][(h+1)/2][(w+1)/2][C]")
    _check(_lib.fwi_pool2_bf16(n, h, w, c, mode, _ptr(x), _ptr(y), _stream(stream)))


def fwi_up2_bf16(x, y, mode=0, stream=None):
    """y [n][ho][wo][C] from x [n][(ho+1)/2][(wo+1)/2][C]: nearest neighbour
    (mode 0) or divided by the block's cell count (mode 1)."""
    _bf16_nhwc(x, "x")
    _bf16_nhwc(y, "y")
    n, ho, wo, c = y.shape
    if tuple(x.shape) != (n, (ho + 1) // 2, (wo + 1) // 2, c):
        raise ValueError("x must be [n][(ho+1)/2][(wo+1)/2][C]")
    _check(_lib.fwi_up2_bf16(n, ho, wo, c, mode, _ptr(x), _ptr(y), _stream(stream)))


def fwi_add_bf16(x, y, z, stream=None):
    for t, name in ((x, "x"), (y, "y"), (z, "z")):
        if t.dtype != torch.bfloat16 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name} must be a contiguous bfloat16 CUDA tensor")
    if not (x.shape == y.shape == z.shape):
        raise ValueError("x, y and z must have one shape")
    _check(_lib.fwi_add_bf16(x.numel(), _ptr(x), _ptr(y), _ptr(z), _stream(stream)))


def fwi_sur_pack(v, G, X, m, in_scale=1.0, in_shift=0.0, stream=None):
    """X [nimg][nx][m][c0] bf16 from models v [nmod][nz][nx] fp32 and the
    geometry channels G [nx][c0] fp32 (see include/fwi.h)."""
    nmod, nz, nx = v.shape
    nimg, c0 = -(-nmod // m), G.shape[1]
    _f32(v, (nmod, nz, nx), "v")
    _f32(G, (nx, c0), "G")
    _bf16_nhwc(X, "X")
    if tuple(X.shape) != (nimg, nx, m, c0):
        raise ValueError(f"X must be {(nimg, nx, m, c0)}")
    _check(_lib.fwi_sur_pack(nmod, m, nz, nx, c0, float(in_scale), float(in_shift), _ptr(v),
                             _ptr(G), _ptr(X), _stream(stream)))


def fwi_sur_unpack_grad(dX, dv, m, in_scale=1.0, stream=None):
    nmod, nz, nx = dv.shape
    nimg, c0 = dX.shape[0], dX.shape[3]
    _f32(dX, (nimg, nx, m, c0), "dX")
    _f32(dv, (nmod, nz, nx), "dv")
    _check(_lib.fwi_sur_unpack_grad(nmod, m, nz, nx, c0, float(in_scale), _ptr(dX), _ptr(dv),
                                    _stream(stream)))


def _int_dev(t, n, name):
    if t.dtype != torch.int32 or t.numel() != n or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous int32 CUDA tensor of {n} entries")


def fwi_sur_traces(Y, d, m, amp, rec_ix, stream=None):
    """d [nmod][ns][nr][nt] = amp sign(y) (e^|y| - 1) from Y [nimg][nx][m][cout]."""
    nmod, ns, nr, nt = d.shape
    nimg, nx, _, cout = Y.shape
    _f32(Y, (nimg, nx, m, cout), "Y")
    _f32(d, (nmod, ns, nr, nt), "d")
    _int_dev(rec_ix, nr, "rec_ix")
    _check(_lib.fwi_sur_traces(nmod, m, ns, nr, nt, nx, cout, float(amp), _ptr(rec_ix), _ptr(Y),
                               _ptr(d), _stream(stream)))


def fwi_sur_output_grad(Y, adj, dY, m, amp, col_rec, scale=1.0, stream=None):
    """dY bf16 [nimg][nx][m][cout]: the trace map's transposed derivative at Y
    applied to adj [nmod][ns][nr][nt]; 0 where no trace reads Y."""
    nmod, ns, nr, nt = adj.shape
    nimg, nx, _, cout = Y.shape
    _f32(Y, (nimg, nx, m, cout), "Y")
    _f32(adj, (nmod, ns, nr, nt), "adj")
    _bf16_nhwc(dY, "dY")
    _int_dev(col_rec, nx, "col_rec")
    _check(_lib.fwi_sur_output_grad(nmod, m, ns, nr, nt, nx, cout, float(amp), float(scale),
                                    _ptr(col_rec), _ptr(Y), _ptr(adj), _ptr(dY),
                                    _stream(stream)))


def fwi_sur_target(d, Yt, m, amp, col_rec, stream=None):
    nmod, ns, nr, nt = d.shape
    nimg, nx, _, cout = Yt.shape
    _f32(d, (nmod, ns, nr, nt), "d")
    _f32(Yt, (nimg, nx, m, cout), "Yt")
    _int_dev(col_rec, nx, "col_rec")
    _check(_lib.fwi_sur_target(nmod, m, ns, nr, nt, nx, cout, float(amp), _ptr(col_rec), _ptr(d),
                               _ptr(Yt), _stream(stream)))


def fwi_sur_loss(Y, Yt, loss, dY, work, stream=None):
    if Y.shape != Yt.shape or tuple(dY.shape) != tuple(Y.shape) or dY.dtype != torch.bfloat16:
        raise ValueError("Y, Yt (fp32) and dY (bf16) must have one shape")
    wp, wf = _work(work)
    _check(_lib.fwi_sur_loss(Y.numel(), _ptr(Y), _ptr(Yt), _ptr(loss), _ptr(dY), wp, wf,
                             _stream(stream)))


def fwi_pool_h_bf16(x, y, mode=0, stream=None):
    """y [n][(h+1)/2][w][C]: mean (mode 0) or sum (mode 1) of row pairs of x."""
    _bf16_nhwc(x, "x")
    _bf16_nhwc(y, "y")
    n, h, w, c = x.shape
    if tuple(y.shape) != (n, (h + 1) // 2, w, c):
        raise ValueError("y must be [n][(h+1)/2][w][C]")
    _check(_lib.fwi_pool_h_bf16(n, h, w, c, mode, _ptr(x), _ptr(y), _stream(stream)))


def fwi_up_h_bf16(x, y, mode=0, stream=None):
    """y [n][ho][w][C] from x [n][(ho+1)/2][w][C]: nearest rows (mode 0), divided
    by the block's rows (mode 1)."""
    _bf16_nhwc(x, "x")
    _bf16_nhwc(y, "y")
    n, ho, w, c = y.shape
    if tuple(x.shape) != (n, (ho + 1) // 2, w, c):
        raise ValueError("x must be [n][(ho+1)/2][w][C]")
    _check(_lib.fwi_up_h_bf16(n, ho, w, c, mode, _ptr(x), _ptr(y), _stream(stream)))


def fwi_sur_weights_prep(W3, Wb, WTb, stream=None):
    cout, _, cin = W3.shape
    _f32(W3, (cout, 3, cin), "W3")
    if tuple(Wb.shape) != (cout, 3, 3, cin) or tuple(WTb.shape) != (cin, 3, 3, cout):
        raise ValueError("Wb [cout][3][3][cin] and WTb [cin][3][3][cout] bf16 needed")
    _check(_lib.fwi_sur_weights_prep(cout, cin, _ptr(W3), _ptr(Wb), _ptr(WTb), _stream(stream)))


def fwi_sur_wgrad_centre(dW, dW3, stream=None):
    cout, _, cin = dW3.shape
    _f32(dW, (cout, 3, 3, cin), "dW")
    _f32(dW3, (cout, 3, cin), "dW3")
    _check(_lib.fwi_sur_wgrad_centre(cout, cin, _ptr(dW), _ptr(dW3), _stream(stream)))


def fwi_rel_error(g, g_ref, err=None, stream=None):
    """err [B] = ||g_b - g_ref_b|| / ||g_ref_b|| per model of g, g_ref [B][...] (fp32,
    device); a zero reference gives 0 for a zero g_b, else inf."""
    B = g.shape[0]
    _f32(g_ref, tuple(g.shape), "g_ref")
    _f32(g, tuple(g.shape), "g")
    if err is None:
        err = torch.empty((B,), dtype=torch.float32, device=g.device)
    _f32(err, (B,), "err")
    _check(_lib.fwi_rel_error(B, g[0].numel(), _ptr(g), _ptr(g_ref), _ptr(err), _stream(stream)))
    return err


def fwi_channel_sum(dP, db, work=None, stream=None):
    c = dP.shape[-1]
    _f32(db, (c,), "db")
    wp, wf = _work(work)
    _check(_lib.fwi_channel_sum(dP.numel() // c, c, _ptr(dP), _ptr(db), wp, wf, _stream(stream)))


def fwi_adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(_lib.fwi_adam_step(param.numel(), float(lr), float(beta1), float(beta2), float(eps),
                              int(step), _ptr(param), _ptr(grad), _ptr(m), _ptr(v),
                              _stream(stream)))


def fwi_conv3x3_weights_prep(W, Wb, WTb, stream=None):
    cout, _, _, cin = W.shape
    _check(_lib.fwi_conv3x3_weights_prep(cout, cin, _ptr(W), _ptr(Wb), _ptr(WTb),
                                         _stream(stream)))


def fwi_time_bias(b, E, phi, out, stream=None):
    _check(_lib.fwi_time_bias(phi.shape[0], b.shape[0], E.shape[1], _ptr(b), _ptr(E), _ptr(phi),
                              _ptr(out), _stream(stream)))


def fwi_time_bias_grad(db, phi_row, dE, stream=None):
    _check(_lib.fwi_time_bias_grad(db.shape[0], phi_row.shape[0], _ptr(db), _ptr(phi_row),
                                   _ptr(dE), _stream(stream)))


def fwi_check(plan, workspace, stream=None):
    _check(_lib.fwi_check(plan.raw, _ptr(workspace), _stream(stream)))


# ----------------------------------------------------------------- convenience plan

class Plan:
    """A plan plus the device buffers it needs, allocated with torch on
    ``device`` (default: the current CUDA device)."""

    def __init__(self, prob: Problem, w2: W2Params | None = None, device=None,
                 snapshots: bool = True):
        self.prob = prob
        self.w2p = w2 or W2Params()
        self.handle = fwi_plan_create(prob, self.w2p)
        self.ws_bytes, self.ctx_bytes, self.snap_bytes = fwi_plan_sizes(self.handle)
        self.kernels = fwi_plan_kernels(self.handle)   # the propagator family it runs
        self.device = torch.device(device) if device is not None else \
            torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.snapshots = torch.empty(self.snap_bytes // 4, dtype=torch.float32,
                                     device=self.device) if snapshots else None

    # shapes
    @property
    def model_shape(self):
        p = self.prob
        return (p.batch, p.nz, p.nx)

    @property
    def data_shape(self):
        p = self.prob
        return (p.batch, p.ns, p.nr, p.nt)

    def new_ctx(self):
        return torch.empty(self.ctx_bytes, dtype=torch.uint8, device=self.device)

    def forward(self, v, d_syn=None, store=True, stream=None):
        """d_syn = F(v); with ``store`` the snapshots for the adjoint are kept."""
        _f32(v, self.model_shape, "v")
        if d_syn is None:
            d_syn = torch.empty(self.data_shape, dtype=torch.float32, device=self.device)
        _f32(d_syn, self.data_shape, "d_syn")
        snap = self.snapshots if store else None
        if store and snap is None:
            raise ValueError("plan was created without a snapshot buffer")
        fwi_forward(self.handle, v, d_syn, snap, self.workspace, stream)
        return d_syn, snap

    def w2_prepare(self, d_obs, ctx=None, stream=None):
        _f32(d_obs, self.data_shape, "d_obs")
        if ctx is None:
            ctx = self.new_ctx()
        fwi_w2_prepare(self.handle, d_obs, ctx, stream)
        return ctx

    def w2_misfit(self, ctx, d_syn, want_w2=True, want_adj=True, stream=None):
        _f32(d_syn, self.data_shape, "d_syn")
        p = self.prob
        J = torch.empty(p.batch, dtype=torch.float32, device=self.device)
        w2 = torch.empty((p.batch, p.ns, p.nr), dtype=torch.float32,
                         device=self.device) if want_w2 else None
        adj = torch.empty(self.data_shape, dtype=torch.float32,
                          device=self.device) if want_adj else None
        fwi_w2_misfit(self.handle, ctx, d_syn, J, w2, adj, self.workspace, stream)
        return J, w2, adj

    def l2_misfit(self, d_obs, d_syn, sigma=1.0, want_adj=True, stream=None):
        """Least-squares potential (J [B], adj or None) of the DPS baseline."""
        _f32(d_obs, self.data_shape, "d_obs")
        _f32(d_syn, self.data_shape, "d_syn")
        J = torch.empty(self.prob.batch, dtype=torch.float32, device=self.device)
        adj = torch.empty(self.data_shape, dtype=torch.float32,
                          device=self.device) if want_adj else None
        fwi_l2_misfit(self.handle, d_obs, d_syn, sigma, J, adj, stream)
        return J, adj

    def adjoint_grad(self, v, adj, grad=None, stream=None):
        _f32(v, self.model_shape, "v")
        _f32(adj, self.data_shape, "adj")
        if grad is None:
            grad = torch.empty(self.model_shape, dtype=torch.float32, device=self.device)
        fwi_adjoint_grad(self.handle, v, adj, self.snapshots, grad, self.workspace, stream)
        return grad

    def gradient(self, v, ctx, stream=None):
        """J(v), dJ/dv and per-trace W2 (forward -> misfit -> adjoint)."""
        d_syn, _ = self.forward(v, stream=stream)
        J, w2, adj = self.w2_misfit(ctx, d_syn, stream=stream)
        grad = self.adjoint_grad(v, adj, stream=stream)
        return J, grad, w2

    def check(self, stream=None):
        fwi_check(self.handle, self.workspace, stream)

    def close(self):
        self.workspace = None
        self.snapshots = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def guided_step(v_prime, v0hat, g, h, params: GuideParams, v_out=None, stream=None):
    """Algorithm 2 update on [B][nz][nx] tensors; returns (v_out, rho [B])."""
    B, nz, nx = v_prime.shape
    for t, n in ((v_prime, "v_prime"), (v0hat, "v0hat"), (g, "g"), (h, "h")):
        _f32(t, (B, nz, nx), n)
    if v_out is None:
        v_out = torch.empty_like(v_prime)
    rho = torch.empty(B, dtype=torch.float32, device=v_prime.device)
    fwi_guided_step(B, nz, nx, params, v_prime, v0hat, g, h, v_out, rho, stream)
    return v_out, rho


def tv_grad(v, g=None, alpha=1.0, unit=1.0, stream=None):
    """(h = g + alpha dTV(v / unit)/dv, TV(v / unit) [B]) on [B][nz][nx] tensors."""
    B, nz, nx = v.shape
    _f32(v, (B, nz, nx), "v")
    if g is not None:
        _f32(g, (B, nz, nx), "g")
    h = torch.empty_like(v)
    tv = torch.empty(B, dtype=torch.float32, device=v.device)
    fwi_tv_grad(B, nz, nx, alpha, unit, v, g, h, tv, stream)
    return h, tv


def image_metrics(v_true, v_rec, data_range, stream=None):
    """[B][3]: relative l2 error, PSNR (dB), SSIM (Sec. 6.3)."""
    B, nz, nx = v_true.shape
    _f32(v_true, (B, nz, nx), "v_true")
    _f32(v_rec, (B, nz, nx), "v_rec")
    out = torch.empty((B, 3), dtype=torch.float32, device=v_true.device)
    fwi_image_metrics(B, nz, nx, data_range, v_true, v_rec, out, stream)
    return out


def autotune(prob: Problem, w2: W2Params | None = None, v=None, trial_steps: int = 64,
             stream=None):
    """The problem with `kernels` and `shape` set to the family and thread
    shape fwi_autotune_kernels measured fastest, and the predicted
    milliseconds of one pass at nt steps
    [resident, tiled, cluster, CPML] (-1: the family cannot run it).  `v`
    ([B][nz][nx] on the device) defaults to the linear v(z) ramp from 1500 m/s
    to min(4500, v_max) m/s; the scratch is a temporary torch buffer."""
    import dataclasses
    w2 = w2 or W2Params()
    if v is None:
        top = min(4500.0, float(prob.v_max))
        z = torch.linspace(0.0, 1.0, prob.nz, device="cuda")
        v = (min(1500.0, top) + (top - min(1500.0, top)) * z)[None, :, None].expand(
            prob.batch, prob.nz, prob.nx).contiguous()
    n = fwi_autotune_scratch_bytes(prob, w2, trial_steps)
    scratch = torch.empty(max(n, 256), dtype=torch.uint8, device=v.device)
    fam, shape, ms, _ = fwi_autotune_kernels(prob, w2, v, trial_steps, scratch, stream)
    return dataclasses.replace(prob, kernels=fam, shape=shape), ms


class Queue:
    """Plans of uneven grid sizes whose forward and adjoint passes each run as
    ONE persistent launch (fwi_queue_forward / fwi_queue_adjoint): every
    (model, shot) unit of every plan on one list, drawn by the CTAs from a
    device counter.  Plans are taken largest first.  ``gradient`` runs the
    queued forward, each plan's W2 misfit, the queued adjoint (with the shot
    sums); outputs are allocated here once and reused."""

    def __init__(self, plans):
        if not 1 <= len(plans) <= FWI_QUEUE_MAX_PLANS:
            raise ValueError(f"1 to {FWI_QUEUE_MAX_PLANS} plans")
        self.plans = list(plans)
        dev = self.plans[0].device
        self.counter = torch.zeros(1, dtype=torch.int32, device=dev)
        f32 = dict(dtype=torch.float32, device=dev)
        self.d_syn = [torch.empty(p.data_shape, **f32) for p in self.plans]
        self.grad = [torch.empty(p.model_shape, **f32) for p in self.plans]

    @staticmethod
    def _arr(ts):
        return (_vp * len(ts))(*[ctypes.cast(_ptr(t), _vp) for t in ts])

    def forward(self, vs, stream=None):
        for p, v in zip(self.plans, vs):
            _f32(v, p.model_shape, "v")
        _check(_lib.fwi_queue_forward((_vp * len(self.plans))(*[p.handle.raw for p in self.plans]),
                                      len(self.plans), self._arr(vs), self._arr(self.d_syn),
                                      self._arr([p.snapshots for p in self.plans]),
                                      self._arr([p.workspace for p in self.plans]),
                                      _ptr(self.counter), _stream(stream)))
        return self.d_syn

    def adjoint(self, vs, adjs, stream=None):
        _check(_lib.fwi_queue_adjoint((_vp * len(self.plans))(*[p.handle.raw for p in self.plans]),
                                      len(self.plans), self._arr(vs), self._arr(adjs),
                                      self._arr([p.snapshots for p in self.plans]),
                                      self._arr(self.grad),
                                      self._arr([p.workspace for p in self.plans]),
                                      _ptr(self.counter), _stream(stream)))
        return self.grad

    def gradient(self, vs, ctxs, stream=None):
        """(J list, dJ/dv list) for models vs[i] against contexts ctxs[i]."""
        self.forward(vs, stream)
        Js, adjs = [], []
        for p, c, d in zip(self.plans, ctxs, self.d_syn):
            J, _, adj = p.w2_misfit(c, d, want_w2=False, stream=stream)
            Js.append(J)
            adjs.append(adj)
        self.adjoint(vs, adjs, stream)
        return Js, self.grad


class Group:
    """Plans of uneven grid sizes whose gradients run as one unit
    (fwi_group_gradient): each plan's forward -> misfit -> adjoint on a stream
    of its own, forked from and joined back to the calling stream, so a CUDA
    graph capture of one call records the whole set.  The Plan objects keep
    their own workspaces and snapshot buffers; outputs are allocated here once
    and reused by every call."""

    def __init__(self, plans):
        self.plans = list(plans)
        raw = (_vp * len(self.plans))(*[p.handle.raw for p in self.plans])
        out = _vp()
        _check(_lib.fwi_group_create(raw, len(self.plans), ctypes.byref(out)))
        self.raw = out
        self.d_syn = [torch.empty(p.data_shape, dtype=torch.float32, device=p.device)
                      for p in self.plans]
        self.adj = [torch.empty_like(d) for d in self.d_syn]
        self.grad = [torch.empty(p.model_shape, dtype=torch.float32, device=p.device)
                     for p in self.plans]
        self.J = [torch.empty(p.prob.batch, dtype=torch.float32, device=p.device)
                  for p in self.plans]

    def gradient(self, vs, ctxs, stream=None):
        """(J list, dJ/dv list) for models vs[i] against observation contexts
        ctxs[i] (from plans[i].w2_prepare)."""
        for p, v in zip(self.plans, vs):
            _f32(v, p.model_shape, "v")
        lists = [
            [_ptr(v) for v in vs], [_ptr(c) for c in ctxs], [_ptr(t) for t in self.d_syn],
            [_ptr(t) for t in self.adj], [_ptr(p.snapshots) for p in self.plans],
            [_ptr(t) for t in self.grad], [_ptr(t) for t in self.J],
            [_ptr(p.workspace) for p in self.plans]]
        arrs = [(_vp * len(lst))(*[ctypes.cast(x, _vp) if x is not None else None for x in lst])
                for lst in lists]
        _check(_lib.fwi_group_gradient(self.raw, *arrs, _stream(stream)))
        return self.J, self.grad

    def close(self):
        if self.raw:
            _lib.fwi_group_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
