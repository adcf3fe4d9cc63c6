"""FP64 oracle of the CPML variant: the absorbing layer as a convolutional
perfectly matched layer instead of the damping sponge (the paper's solver
absorbs with a PML, Sec. 6.1; this is the reading of it listed with the
variants).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
It shares no code with the CUDA binding.  numpy + scipy.sparse, plain and
slow: every spatial operator is an explicit sparse matrix, and the adjoint
solve uses their transposes (``.T``), so it is the exact transpose of the
forward by construction.

Equations (per shot; 4th-order stencils, zero values outside the padded
grid on all four sides, i.e. top_bc = 0 only).  With the layer's stretching
s_x = 1 + sigma_x / (i omega) on the left/right columns and s_z on the
bottom rows, the Laplacian becomes d/dx (1/s_x) d/dx (1/s_x) u + (z), and
each 1/s_x convolution is a memory variable updated once per step:

    psi_x^n  = b_x psi_x^{n-1}  + a_x (Dx u^n)
    h_x^n    = Dxx u^n + Dx psi_x^n
    zeta_x^n = b_x zeta_x^{n-1} + a_x h_x^n                (same in z)
    B^n      = h_x + zeta_x + h_z + zeta_z + s^n
    u^{n+1}  = 2 u^n - u^{n-1} + kappa B^n,   kappa = v_pad^2 dt^2

with b = exp(-sigma dt), a = b - 1, sigma(d) = d0 (d/nb)^2 in the d-th cell
into the layer (d as in the sponge: 0 inside the physical grid), and
d0 = 3 v_ref ln(1/R) / (2 nb h) per direction (h = dx or dz).  Dx is the
4th-order central first difference (1, -8, 0, 8, -1)/(12 dx), Dxx the
4th-order second difference.  Source s^n = f(n dt)/(dx dz) at the source
cell; sample n records u^{n+1}.  With sigma = 0 (refl_R = 1) the scheme is
exactly the undamped leapfrog of the sponge oracle.

Gradient: dJ/dv_pad = 2 v_pad dt^2 sum_n mu^{n+1} B^n, mu the adjoint of u.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import oracle as O


def _d1(n, h):
    """1D 4th-order central first difference, zero outside [0, n)."""
    return sp.diags([1.0, -8.0, 8.0, -1.0], [-2, -1, 1, 2], shape=(n, n)) / (12.0 * h)


def _d2(n, h):
    """1D 4th-order second difference, zero outside [0, n)."""
    return sp.diags([-1.0 / 12, 4.0 / 3, -5.0 / 2, 4.0 / 3, -1.0 / 12], [-2, -1, 0, 1, 2],
                    shape=(n, n)) / (h * h)


def operators(prob: O.Problem):
    """Sparse Dx, Dz, Dxx, Dzz on the padded grid flattened row-major
    (index z * NX + x)."""
    NZ, NX = prob.NZ, prob.NX
    Iz, Ix = sp.identity(NZ), sp.identity(NX)
    Dx = sp.kron(Iz, _d1(NX, prob.dx)).tocsr()
    Dz = sp.kron(_d1(NZ, prob.dz), Ix).tocsr()
    Dxx = sp.kron(Iz, _d2(NX, prob.dx)).tocsr()
    Dzz = sp.kron(_d2(NZ, prob.dz), Ix).tocsr()
    return Dx, Dz, Dxx, Dzz


def profiles(prob: O.Problem):
    """(a_x, b_x, a_z, b_z) on the padded grid [NZ][NX] (a = b - 1)."""
    NZ, NX, nb, nx, nz = prob.NZ, prob.NX, prob.nb, prob.nx, prob.nz
    lnR = np.log(1.0 / prob.refl_R)
    px, pz = np.arange(NX), np.arange(NZ)
    cx = np.where(px < nb, nb - px, np.where(px > nb + nx - 1, px - (nb + nx - 1), 0)).astype(float)
    cz = np.where(pz > nz - 1, pz - (nz - 1), 0).astype(float)
    if nb > 0:
        sx = 3.0 * prob.v_ref * lnR / (2.0 * nb * prob.dx) * (cx / nb) ** 2
        sz = 3.0 * prob.v_ref * lnR / (2.0 * nb * prob.dz) * (cz / nb) ** 2
    else:
        sx, sz = np.zeros(NX), np.zeros(NZ)
    bx, bz = np.exp(-sx * prob.dt), np.exp(-sz * prob.dt)
    BX = np.broadcast_to(bx[None, :], (NZ, NX))
    BZ = np.broadcast_to(bz[:, None], (NZ, NX))
    return BX - 1.0, BX.copy(), BZ - 1.0, BZ.copy()


def _cells(prob: O.Problem, s: int):
    NX = prob.NX
    src = int(prob.src_iz[s]) * NX + int(prob.src_ix[s]) + prob.nb
    rec = np.asarray(prob.rec_iz, dtype=np.int64) * NX + np.asarray(prob.rec_ix) + prob.nb
    return src, rec


def forward_shot(prob: O.Problem, v, s: int, keep_record: bool = False, wavelet=None):
    """d [nr][nt] (and the record B^n [nt][NZ*NX] when asked)."""
    assert prob.top_bc == 0 and prob.space_order == 4
    Dx, Dz, Dxx, Dzz = operators(prob)
    ax, bx, az, bz = (p.ravel() for p in profiles(prob))
    kappa = (O.pad_model(prob, v) * prob.dt).ravel() ** 2
    f = O.ricker_series(prob) if wavelet is None else np.asarray(wavelet, dtype=float)
    src, rec = _cells(prob, s)
    n = prob.NZ * prob.NX
    u, up = np.zeros(n), np.zeros(n)
    psx, psz, zex, zez = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    d = np.empty((len(rec), prob.nt))
    Brec = np.empty((prob.nt, n)) if keep_record else None
    for k in range(prob.nt):
        psx = bx * psx + ax * (Dx @ u)
        psz = bz * psz + az * (Dz @ u)
        hx = Dxx @ u + Dx @ psx
        hz = Dzz @ u + Dz @ psz
        zex = bx * zex + ax * hx
        zez = bz * zez + az * hz
        B = hx + hz + zex + zez
        B[src] += f[k] / (prob.dx * prob.dz)
        un = 2.0 * u - up + kappa * B
        d[:, k] = un[rec]
        if keep_record:
            Brec[k] = B
        up, u = u, un
    return d, Brec


def adjoint_shot(prob: O.Problem, v, s: int, adj, Brec) -> np.ndarray:
    """dJ/dv_pad [NZ][NX] for the adjoint source adj [nr][nt] (= dJ/dd):
    reverse-mode of forward_shot, step by step, with transposed operators."""
    Dx, Dz, Dxx, Dzz = operators(prob)
    DxT, DzT, DxxT, DzzT = Dx.T.tocsr(), Dz.T.tocsr(), Dxx.T.tocsr(), Dzz.T.tocsr()
    ax, bx, az, bz = (p.ravel() for p in profiles(prob))
    vpad = O.pad_model(prob, v).ravel()
    kappa = (vpad * prob.dt) ** 2
    _, rec = _cells(prob, s)
    n = prob.NZ * prob.NX
    adj = np.asarray(adj, dtype=float)
    g_kappa = np.zeros(n)
    mu1 = np.zeros(n)      # adjoint of u^{k+1} (being completed)
    mu0 = np.zeros(n)      # adjoint of u^k (accumulating)
    psbx, psbz, zebx, zebz = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    for k in range(prob.nt - 1, -1, -1):
        np.add.at(mu1, rec, adj[:, k])                 # d^k = R u^{k+1}
        # u^{k+1} = 2 u^k - u^{k-1} + kappa B^k
        Bb = kappa * mu1
        g_kappa += mu1 * Brec[k]
        mu0 += 2.0 * mu1
        mum = -mu1                                     # into the adjoint of u^{k-1}
        # B = h_x + zeta_x + h_z + zeta_z + s
        zebx += Bb
        zebz += Bb
        hbx = Bb + ax * zebx                           # zeta^k = b zeta^{k-1} + a h
        hbz = Bb + az * zebz
        zebx *= bx
        zebz *= bz
        # h = Dxx u^k + Dx psi^k
        mu0 += DxxT @ hbx + DzzT @ hbz
        psbx += DxT @ hbx
        psbz += DzT @ hbz
        # psi^k = b psi^{k-1} + a Dx u^k
        mu0 += DxT @ (ax * psbx) + DzT @ (az * psbz)
        psbx *= bx
        psbz *= bz
        mu1, mu0 = mu0, mum
    return (2.0 * vpad * prob.dt ** 2 * g_kappa).reshape(prob.NZ, prob.NX)


def forward(prob: O.Problem, v) -> np.ndarray:
    """d_syn [B][ns][nr][nt] for models v [B][nz][nx]."""
    v = np.asarray(v, dtype=float)
    return np.stack([np.stack([forward_shot(prob, v[b], s)[0] for s in range(prob.ns)])
                     for b in range(v.shape[0])])


def gradient(prob: O.Problem, v, ctx: O.ObsContext, w2p: O.W2Params):
    """J [B], dJ/dv [B][nz][nx] of Eq. final_objective with CPML solves: the
    misfit and its adjoint source come from the sponge oracle's W2 code."""
    v = np.asarray(v, dtype=float)
    B = v.shape[0]
    d = np.empty((B, prob.ns, prob.nr, prob.nt))
    recs = {}
    for b in range(B):
        for s in range(prob.ns):
            d[b, s], recs[b, s] = forward_shot(prob, v[b], s, keep_record=True)
    J, _, adj = O.w2_misfit(ctx, d, prob.dt, w2p, True)
    g = np.zeros((B, prob.nz, prob.nx))
    for b in range(B):
        for s in range(prob.ns):
            g[b] += O.fold(prob, adjoint_shot(prob, v[b], s, adj[b, s], recs[b, s]))
    return J, g
