"""Python driver for the FP64 CPU oracle (``fwi_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It does
not import the CUDA binding and shares no code with it.

The C functions are single-threaded; this module runs independent
(model, shot) units on a thread pool (ctypes releases the GIL during a call).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fwi.so")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source (plain gcc,
    no machine-specific flags, no FMA contraction so that x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_lib_lock = threading.Lock()


def lib():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        L = ctypes.CDLL(build())
        i, d = ctypes.c_int, ctypes.c_double
        L.orc_ricker.restype = d
        L.orc_ricker.argtypes = [d, d, d]
        L.orc_ricker_series.argtypes = [i, d, d, d, _dp]
        L.orc_pad_model.argtypes = [i, i, i, _dp, _dp]
        L.orc_fold_add.argtypes = [i, i, i, _dp, _dp]
        L.orc_damping.argtypes = [i, i, i, d, d, d, d, _dp]
        L.orc_laplacian.argtypes = [i, i, d, d, i, i, _dp, _dp]
        L.orc_laplacian_T.argtypes = [i, i, d, d, i, i, _dp, _dp]
        L.orc_forward_shot.argtypes = [i, i, i, i, i, d, d, d, _dp, _dp, _dp, i, i,
                                       i, _ip, _ip, _dp, _dp]
        L.orc_adjoint_shot.argtypes = [i, i, i, i, i, d, d, d, _dp, _dp, _dp, i, i,
                                       i, _ip, _ip, _dp, _dp, _dp]
        L.orc_cdf.argtypes = [i, d, d, _dp, _dp, _dp, _dp]
        L.orc_quantiles.argtypes = [i, d, i, _dp, _dp, _ip]
        L.orc_w2_from_quantiles.restype = d
        L.orc_w2_from_quantiles.argtypes = [i, _dp, _dp]
        L.orc_w2_signals.restype = d
        L.orc_w2_signals.argtypes = [i, d, d, i, _dp, _dp]
        L.orc_w2_prepare.restype = d
        L.orc_w2_prepare.argtypes = [i, i, d, d, d, d, i, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_w2_misfit.restype = d
        L.orc_w2_misfit.argtypes = [i, i, d, d, i, _dp, _dp, _dp, _dp, d, i, _dp, _dp]
        L.orc_l2_misfit.restype = d
        L.orc_l2_misfit.argtypes = [ctypes.c_long, d, _dp, _dp, _dp]
        L.orc_tv_grad.restype = d
        L.orc_tv_grad.argtypes = [i, i, d, d, _dp, _dp, _dp]
        L.orc_image_metrics.argtypes = [i, i, d, _dp, _dp, _dp]
        L.orc_guided_step.restype = d
        L.orc_guided_step.argtypes = [i, i, d, d, d, d, d, d, d, _dp, _dp, _dp, _dp, _dp]
        _lib = L
        return _lib


def _p(a):
    """ctypes pointer to a C-contiguous float64/int32 array (or None)."""
    if a is None:
        return None
    if a.dtype == np.float64:
        assert a.flags.c_contiguous
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int32:
        assert a.flags.c_contiguous
        return a.ctypes.data_as(_ip)
    raise TypeError(a.dtype)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass
class Problem:
    """Discretisation and acquisition of Sec. 2.1 / 6.1 (see fwi_oracle.c header)."""
    nz: int
    nx: int
    nb: int
    nt: int
    dz: float
    dx: float
    dt: float
    src_iz: tuple
    src_ix: tuple
    rec_iz: tuple
    rec_ix: tuple
    f_peak: float = 15.0
    t0: float | None = None
    v_ref: float = 4500.0
    refl_R: float = 1e-3
    top_bc: int = 0
    space_order: int = 4      # 4 (the hot path) or 8 (the paper's solver, Sec. 6.1)

    @property
    def NZ(self):
        return self.nz + self.nb

    @property
    def NX(self):
        return self.nx + 2 * self.nb

    @property
    def ns(self):
        return len(self.src_ix)

    @property
    def nr(self):
        return len(self.rec_ix)

    @property
    def t0_(self):
        return 1.1 / self.f_peak if self.t0 is None else self.t0


@dataclasses.dataclass
class W2Params:
    """Misfit hyperparameters: k (Eq. omega_def, Sec. 6.3 k = 100), the c' factor
    1.1 and eps' = 1e-9 (Sec. 6.2), N_xi = 1000 (Sec. 6.2)."""
    k: float = 100.0
    cshift_factor: float = 1.1
    eps_density: float = 1e-9
    n_xi: int = 1000
    # False: J = sum W2 / S_obs (Eq. final_objective); True: the raw baseline
    # J = sum W2^2 / sum int |Q_obs|^2 (Sec. 6.3, Baseline 1; use with k = 0)
    squared: bool = False


@dataclasses.dataclass
class GuideParams:
    """Eq. rho / Eq. kappa hyperparameters (Sec. 6.3: c = 0.1, tau = 0, eps = 1e-4)."""
    rho0: float = 1.0
    c: float = 0.1
    tau: float = 0.0
    gamma: float = 0.5
    eps: float = 1e-4
    kappa_min: float = 0.0
    kappa_max: float = 0.0


def nthreads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


# --------------------------------------------------------------------------- pieces

def ricker_series(prob: Problem) -> np.ndarray:
    f = np.empty(prob.nt)
    lib().orc_ricker_series(prob.nt, prob.dt, prob.f_peak, prob.t0_, _p(f))
    return f


def pad_model(prob: Problem, v) -> np.ndarray:
    v = _f64(v)
    out = np.empty((prob.NZ, prob.NX))
    lib().orc_pad_model(prob.nz, prob.nx, prob.nb, _p(v), _p(out))
    return out


def fold(prob: Problem, gpad) -> np.ndarray:
    gpad = _f64(gpad)
    g = np.zeros((prob.nz, prob.nx))
    lib().orc_fold_add(prob.nz, prob.nx, prob.nb, _p(gpad), _p(g))
    return g


def damping(prob: Problem) -> np.ndarray:
    eta = np.empty((prob.NZ, prob.NX))
    lib().orc_damping(prob.nz, prob.nx, prob.nb, prob.dz, prob.dx, prob.v_ref,
                      prob.refl_R, _p(eta))
    return eta


def laplacian(u, dz, dx, top_bc=0, transpose=False, order=4) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    fn = lib().orc_laplacian_T if transpose else lib().orc_laplacian
    fn(u.shape[0], u.shape[1], dz, dx, top_bc, order, _p(u), _p(out))
    return out


def _rec_arrays(prob: Problem):
    rz = np.ascontiguousarray(prob.rec_iz, dtype=np.int32)
    rx = np.ascontiguousarray(np.asarray(prob.rec_ix) + prob.nb, dtype=np.int32)
    return rz, rx


def forward_shot(prob: Problem, v, s: int, keep_wavefield: bool = False,
                 wavelet=None, rec=None):
    """One shot of Eq. (1).  Returns (d [nr][nt], u_all or None).

    ``wavelet`` overrides the Ricker series; ``rec`` = (rz, rx) padded-grid
    receiver cells overriding the surface receivers."""
    vpad = pad_model(prob, v)
    eta = damping(prob)
    f = ricker_series(prob) if wavelet is None else _f64(wavelet)
    rz, rx = _rec_arrays(prob) if rec is None else (np.ascontiguousarray(rec[0], dtype=np.int32),
                                                    np.ascontiguousarray(rec[1], dtype=np.int32))
    d = np.empty((len(rz), prob.nt))
    u_all = np.empty((prob.nt + 1, prob.NZ, prob.NX)) if keep_wavefield else None
    lib().orc_forward_shot(prob.NZ, prob.NX, prob.top_bc, prob.space_order, prob.nt, prob.dz,
                           prob.dx, prob.dt,
                           _p(vpad), _p(eta), _p(f), int(prob.src_iz[s]),
                           int(prob.src_ix[s]) + prob.nb, len(rz), _p(rz), _p(rx),
                           _p(d), _p(u_all))
    return d, u_all


def adjoint_shot(prob: Problem, v, s: int, adj, u_all, wavelet=None, rec=None) -> np.ndarray:
    """Discrete adjoint of one shot: dJ/dv_pad [NZ][NX] for adjoint source adj [nr][nt]."""
    vpad = pad_model(prob, v)
    eta = damping(prob)
    f = ricker_series(prob) if wavelet is None else _f64(wavelet)
    rz, rx = _rec_arrays(prob) if rec is None else (np.ascontiguousarray(rec[0], dtype=np.int32),
                                                    np.ascontiguousarray(rec[1], dtype=np.int32))
    adj = _f64(adj)
    g = np.empty((prob.NZ, prob.NX))
    lib().orc_adjoint_shot(prob.NZ, prob.NX, prob.top_bc, prob.space_order, prob.nt, prob.dz,
                           prob.dx, prob.dt,
                           _p(vpad), _p(eta), _p(f), int(prob.src_iz[s]),
                           int(prob.src_ix[s]) + prob.nb, len(rz), _p(rz), _p(rx),
                           _p(adj), _p(_f64(u_all)), _p(g))
    return g


def cdf(y, dt, eps):
    y = _f64(y)
    p, F, Z = np.empty_like(y), np.empty_like(y), ctypes.c_double()
    lib().orc_cdf(len(y), dt, eps, _p(y), _p(p), _p(F), ctypes.byref(Z))
    return p, F, Z.value


def quantiles(F, dt, nxi):
    F = _f64(F)
    Q = np.empty(nxi)
    ks = np.empty(nxi, dtype=np.int32)
    lib().orc_quantiles(len(F), dt, nxi, _p(F), _p(Q), _p(ks))
    return Q, ks


def w2_signals(ya, yb, dt, eps=1e-9, nxi=1000) -> float:
    ya, yb = _f64(ya), _f64(yb)
    return lib().orc_w2_signals(len(ya), dt, eps, nxi, _p(ya), _p(yb))


# --------------------------------------------------------------------------- W2 over data cubes

@dataclasses.dataclass
class ObsContext:
    omega: np.ndarray     # [B][ns][nr][nt]
    cshift: np.ndarray    # [B][ns][nr]
    Qobs: np.ndarray      # [B][ns][nr][nxi]
    s_tr: np.ndarray      # [B][ns][nr]
    S_obs: np.ndarray     # [B]
    M: np.ndarray         # [B]
    S2: np.ndarray = None  # [B] sum of s_tr^2 (denominator of the squared objective)


def w2_prepare(d_obs, dt, w2p: W2Params) -> ObsContext:
    d_obs = _f64(d_obs)
    B, ns, nr, nt = d_obs.shape
    ntr = ns * nr
    om = np.empty_like(d_obs)
    cs = np.empty((B, ns, nr))
    Q = np.empty((B, ns, nr, w2p.n_xi))
    s_tr = np.empty((B, ns, nr))
    S = np.empty(B)
    M = np.empty(B)
    for b in range(B):
        m = ctypes.c_double()
        S[b] = lib().orc_w2_prepare(ntr, nt, dt, w2p.k, w2p.cshift_factor, w2p.eps_density,
                                    w2p.n_xi, _p(d_obs[b]), _p(om[b]), _p(cs[b]), _p(Q[b]),
                                    _p(s_tr[b]), ctypes.byref(m))
        M[b] = m.value
    return ObsContext(om, cs, Q, s_tr, S, M, (s_tr ** 2).sum(axis=(1, 2)))


def _denominator(ctx: ObsContext, w2p: W2Params, b: int) -> float:
    return float(ctx.S2[b] if w2p.squared else ctx.S_obs[b])


def w2_misfit(ctx: ObsContext, d_syn, dt, w2p: W2Params, with_adjoint=True):
    """Returns (J [B], w2 [B][ns][nr], adj [B][ns][nr][nt] or None)."""
    d_syn = _f64(d_syn)
    B, ns, nr, nt = d_syn.shape
    J = np.empty(B)
    w2 = np.empty((B, ns, nr))
    adj = np.empty_like(d_syn) if with_adjoint else None
    for b in range(B):
        J[b] = lib().orc_w2_misfit(ns * nr, nt, dt, w2p.eps_density, w2p.n_xi, _p(d_syn[b]),
                                   _p(ctx.omega[b]), _p(ctx.cshift[b]), _p(ctx.Qobs[b]),
                                   _denominator(ctx, w2p, b), int(w2p.squared), _p(w2[b]),
                                   _p(adj[b]) if with_adjoint else None)
    return J, w2, adj


# --------------------------------------------------------------------------- whole pipeline

def forward(prob: Problem, v, threads: int | None = None) -> np.ndarray:
    """d_syn [B][ns][nr][nt] for models v [B][nz][nx]."""
    v = _f64(v)
    B = v.shape[0]
    out = np.empty((B, prob.ns, prob.nr, prob.nt))

    def unit(bs):
        b, s = bs
        out[b, s] = forward_shot(prob, v[b], s)[0]

    with ThreadPoolExecutor(threads or nthreads()) as ex:
        list(ex.map(unit, [(b, s) for b in range(B) for s in range(prob.ns)]))
    return out


def gradient(prob: Problem, v, ctx: ObsContext, w2p: W2Params, threads: int | None = None,
             units=None):
    """J [B] and dJ/dv [B][nz][nx] of Eq. final_objective at models v.

    Every (model, shot) unit is independent once the observation context
    exists (the adjoint source of a trace depends only on that trace, c', Q_obs
    and S_obs), so each unit runs forward -> misfit -> adjoint on its own.
    ``units`` restricts the work to a list of (b, s) pairs (used to time a
    bounded sample); the returned arrays then only hold those contributions."""
    v = _f64(v)
    B = v.shape[0]
    if units is None:
        units = [(b, s) for b in range(B) for s in range(prob.ns)]
    Jp = np.zeros((B, prob.ns))
    gp = np.zeros((B, prob.ns, prob.nz, prob.nx))
    w2 = np.zeros((B, prob.ns, prob.nr))

    def unit(bs):
        b, s = bs
        d, u_all = forward_shot(prob, v[b], s, keep_wavefield=True)
        adj = np.empty_like(d)
        Jp[b, s] = lib().orc_w2_misfit(prob.nr, prob.nt, prob.dt, w2p.eps_density, w2p.n_xi,
                                       _p(d), _p(_f64(ctx.omega[b, s])), _p(_f64(ctx.cshift[b, s])),
                                       _p(_f64(ctx.Qobs[b, s])), _denominator(ctx, w2p, b),
                                       int(w2p.squared), _p(w2[b, s]), _p(adj))
        gpad = adjoint_shot(prob, v[b], s, adj, u_all)
        gp[b, s] = fold(prob, gpad)

    with ThreadPoolExecutor(threads or nthreads()) as ex:
        list(ex.map(unit, units))
    J = Jp.sum(axis=1)
    g = gp.sum(axis=1)
    return J, g, w2


def guided_step(vprime, v0hat, g, h, gp: GuideParams):
    """Algorithm 2 update for a batch [B][nz][nx].  Returns (v_out, rho [B])."""
    vprime, v0hat, g, h = map(_f64, (vprime, v0hat, g, h))
    B, nz, nx = vprime.shape
    vout = np.empty_like(vprime)
    rho = np.empty(B)
    for b in range(B):
        rho[b] = lib().orc_guided_step(nz, nx, gp.rho0, gp.c, gp.tau, gp.gamma, gp.eps,
                                       gp.kappa_min, gp.kappa_max, _p(vprime[b]), _p(v0hat[b]),
                                       _p(g[b]), _p(h[b]), _p(vout[b]))
    return vout, rho


# --------------------------------------------------------------------------- baselines, measures

def l2_misfit(d_obs, d_syn, sigma=1.0):
    """Least-squares potential per instance: (J [B], adj [B][...])."""
    d_obs, d_syn = _f64(d_obs), _f64(d_syn)
    B = d_syn.shape[0]
    n = d_syn[0].size
    J = np.empty(B)
    adj = np.empty_like(d_syn)
    for b in range(B):
        J[b] = lib().orc_l2_misfit(n, float(sigma) ** 2, _p(d_obs[b]), _p(d_syn[b]), _p(adj[b]))
    return J, adj


def tv_grad(v, g, alpha, unit=1.0):
    """(TV of v / unit [B], h = g + alpha dTV(v / unit)/dv [B][nz][nx])."""
    v = _f64(v)
    g = _f64(g) if g is not None else np.zeros_like(v)
    B, nz, nx = v.shape
    h = np.empty_like(v)
    tv = np.empty(B)
    for b in range(B):
        tv[b] = lib().orc_tv_grad(nz, nx, float(alpha), float(unit), _p(v[b]), _p(g[b]), _p(h[b]))
    return tv, h


def image_metrics(v_true, v_rec, data_range):
    """[B][3]: relative l2 error, PSNR (dB), SSIM."""
    vt, vr = _f64(v_true), _f64(v_rec)
    B, nz, nx = vt.shape
    out = np.empty((B, 3))
    for b in range(B):
        lib().orc_image_metrics(nz, nx, float(data_range), _p(vt[b]), _p(vr[b]), _p(out[b]))
    return out
