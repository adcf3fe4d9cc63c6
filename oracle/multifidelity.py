"""FP64 oracle of the low-fidelity guidance surrogate: the W2 potential
evaluated on a grid coarsened by two in space and time, the multi-fidelity
route to cheaper physics guidance (Sec. 7), used for the early reverse steps
of Algorithm 2.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product path.
numpy in float64.

Readings:
* Restriction R: coarse cell (I, J) is the mean of the fine cells
  (2I..2I+1, 2J..2J+1) that exist (ceil(nz/2) x ceil(nx/2) coarse cells; an
  odd last row or column averages fewer cells).
* The surrogate potential is Phi_c(R v) with Phi_c the W2 objective of the
  coarse problem (dx, dz and dt doubled, every other receiver, every other
  time sample of the observations, sources at the coarse cells ix // 2); its
  gradient with respect to the fine model is R^T grad Phi_c: each fine cell
  receives its coarse cell's gradient divided by the number of fine cells
  averaged there.
* Decimation D: d_c[b][s][r][m] = d[b][s][2 r][2 m + 1], m < nt // 2: fine sample n
  records the field at t = (n + 1) dt and coarse sample m at (m + 1) 2 dt, so
  sample 2 m + 1 is the one at the same time.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def coarse_shape(nz: int, nx: int):
    return (nz + 1) // 2, (nx + 1) // 2


def restrict(v):
    """R: [B][nz][nx] -> [B][ceil(nz/2)][ceil(nx/2)], mean over each 2 x 2 block."""
    v = np.asarray(v, dtype=np.float64)
    B, nz, nx = v.shape
    nzc, nxc = coarse_shape(nz, nx)
    out = np.zeros((B, nzc, nxc))
    for I in range(nzc):
        for J in range(nxc):
            block = v[:, 2 * I:2 * I + 2, 2 * J:2 * J + 2]
            out[:, I, J] = block.reshape(B, -1).mean(axis=1)
    return out


def restrict_transpose(g, nz: int, nx: int):
    """R^T: [B][nzc][nxc] -> [B][nz][nx]; fine cell (i, j) gets g[i // 2][j // 2] / count."""
    g = np.asarray(g, dtype=np.float64)
    B = g.shape[0]
    out = np.zeros((B, nz, nx))
    for i in range(nz):
        for j in range(nx):
            cnt = (min(2 * (i // 2) + 2, nz) - 2 * (i // 2)) * (min(2 * (j // 2) + 2, nx) - 2 * (j // 2))
            out[:, i, j] = g[:, i // 2, j // 2] / cnt
    return out


def decimate(d):
    """D: [B][ns][nr][nt] -> [B][ns][ceil(nr/2)][nt // 2], even receivers, samples 2 m + 1."""
    d = np.asarray(d, dtype=np.float64)
    nt = d.shape[3]
    return d[:, :, ::2, 1:2 * (nt // 2):2]


def coarse_problem(prob: O.Problem) -> O.Problem:
    """The coarse twin of a problem: grid, spacing and time step doubled,
    sources at ix // 2, receivers the even fine receivers mapped to ix // 2."""
    nzc, nxc = coarse_shape(prob.nz, prob.nx)
    rec = [(int(z) // 2, int(x) // 2) for k, (z, x) in enumerate(zip(prob.rec_iz, prob.rec_ix))
           if k % 2 == 0]
    return O.Problem(nz=nzc, nx=nxc, nb=(prob.nb + 1) // 2, nt=prob.nt // 2,
                     dz=2 * prob.dz, dx=2 * prob.dx, dt=2 * prob.dt,
                     src_iz=[int(z) // 2 for z in prob.src_iz],
                     src_ix=[int(x) // 2 for x in prob.src_ix],
                     rec_iz=[r[0] for r in rec], rec_ix=[r[1] for r in rec],
                     f_peak=prob.f_peak, t0=prob.t0, v_ref=prob.v_ref, refl_R=prob.refl_R,
                     top_bc=prob.top_bc)


def surrogate_potential(prob: O.Problem, d_obs, w2p: O.W2Params, threads=None):
    """Phi_c(R v) and its gradient R^T grad Phi_c for fine models v [B][nz][nx]."""
    cp = coarse_problem(prob)
    ctx = O.w2_prepare(decimate(d_obs), cp.dt, w2p)

    def f(v):
        J, gc, _ = O.gradient(cp, restrict(v), ctx, w2p, threads=threads)
        return J, restrict_transpose(gc, prob.nz, prob.nx)

    return f
