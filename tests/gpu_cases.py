"""Shared case builders for the GPU parity tests: the same seeded inputs are
handed to the CUDA path (through the C ABI binding) and to the FP64 oracle."""
import numpy as np

from oracle import oracle as O
from paper_2603_16393_gb300 import inputs as I

# Tolerances stated for the hot path: seismograms rel-L2 <= 1e-5 (FP32 vs FP64),
# gradients rel-L2 <= 1e-4; the misfit value and its adjoint source follow the
# same split (value 1e-5 relative, adjoint source 1e-4 rel-L2).
TOL_DATA = 1e-5
TOL_J = 1e-5
TOL_ADJ = 1e-4
TOL_GRAD = 1e-4
# End to end through W2 where the quantile map is ill-conditioned (long or
# reverberant traces): a float32-level data difference can move an adjoint
# source by ~1e-3 (interpolated quantiles change bracket), so gradients are
# held to this bound there while every stage keeps its own bar above.
TOL_GRAD_W2 = 5e-3


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problems(nz, nx, nb, nt, ns, batch, nr=None, f_peak=15.0, top_bc=0, v_ref=4500.0,
             v_max=4500.0, dx=10.0, dt=1e-3, geo=None):
    from paper_2603_16393_gb300 import api
    geo = geo or I.surface_geometry(nx, ns, nr)
    gp = api.Problem(nz=nz, nx=nx, nb=nb, nt=nt, dz=dx, dx=dx, dt=dt, src_iz=geo.src_iz,
                     src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, f_peak=f_peak,
                     v_ref=v_ref, v_max=v_max, batch=batch, top_bc=top_bc)
    op = O.Problem(nz=nz, nx=nx, nb=nb, nt=nt, dz=dx, dx=dx, dt=dt, src_iz=geo.src_iz,
                   src_ix=geo.src_ix, rec_iz=geo.rec_iz, rec_ix=geo.rec_ix, f_peak=f_peak,
                   v_ref=v_ref, top_bc=top_bc)
    return gp, op


def models(kind, seeds, nz, nx, scale=1.0, offset=0.0):
    """Velocity models as float32-representable float64 arrays (the GPU sees
    exactly the values the oracle sees)."""
    v = I.model_batch(kind, seeds, nz, nx) * scale + offset
    return v.astype(np.float32).astype(np.float64)


def initial(B, nz, nx, scale=1.0, offset=0.0):
    v = np.stack([I.linear_initial_model(nz, nx)] * B) * scale + offset
    return v.astype(np.float32).astype(np.float64)
