"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method (no wave propagation, no misfit,
no gradient): only velocity models, acquisition geometry and noise drawn from
fixed seeds.  They stand in for the OpenFWI and Marmousi2 velocity models the
paper uses (Sec. 6, "Test datasets"), which are not available: 70x70 grids at
10 m spacing with velocities in 1500-4500 m/s, layered, curved and faulted.

Nothing here imports the CUDA binding or the oracle.
"""
from __future__ import annotations

import dataclasses

import numpy as np

V_MIN = 1500.0
V_MAX = 4500.0


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Surface acquisition on the physical grid (row = depth index z).

    src_iz/src_ix: one source cell per shot; rec_iz/rec_ix: receivers shared by
    all shots (Sec. 6, "Acquisition geometry and discretization").
    """
    src_iz: tuple
    src_ix: tuple
    rec_iz: tuple
    rec_ix: tuple

    @property
    def ns(self) -> int:
        return len(self.src_ix)

    @property
    def nr(self) -> int:
        return len(self.rec_ix)


def surface_geometry(nx: int, ns: int, nr: int | None = None) -> Geometry:
    """ns sources equally spaced on the surface, ix_s = round(j (nx-1)/(ns-1));
    nr receivers at every surface cell 0..nr-1 (default nr = nx)."""
    if nr is None:
        nr = nx
    if ns == 1:
        sx = (nx // 2,)
    else:
        sx = tuple(int(round(j * (nx - 1) / (ns - 1))) for j in range(ns))
    return Geometry(src_iz=(0,) * ns, src_ix=sx,
                    rec_iz=(0,) * nr, rec_ix=tuple(range(nr)))


def layered_model(seed: int, nz: int = 70, nx: int = 70, nlayers: int = 4) -> np.ndarray:
    """Flat-layered model: nlayers-1 distinct interface depths drawn in
    [8, nz-8], sorted velocities in [1500, 4500] with the top layer at 1500 and
    the bottom layer at 4500.  Returns float64 [nz][nx]."""
    rng = np.random.default_rng(seed)
    lo, hi = min(8, nz // 4), max(nz - 8, nz // 4 + nlayers)
    depths = np.sort(rng.choice(np.arange(lo, hi + 1), size=nlayers - 1, replace=False))
    vel = np.sort(rng.uniform(V_MIN, V_MAX, size=nlayers))
    vel[0], vel[-1] = V_MIN, V_MAX
    v = np.empty((nz, nx))
    edges = [0, *depths.tolist(), nz]
    for i in range(nlayers):
        v[edges[i]:edges[i + 1], :] = vel[i]
    return v


def curved_faulted_model(seed: int, nz: int = 70, nx: int = 70) -> np.ndarray:
    """3-5 layers with sinusoidal interfaces z = z0 + a sin(2 pi x / lam + phi)
    and one fault of random dip and throw.  Returns float64 [nz][nx]."""
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(3, 6))
    z0 = np.sort(rng.uniform(0.12 * nz, 0.9 * nz, size=nl - 1))
    amp = rng.uniform(0.0, 0.06 * nz, size=nl - 1)
    lam = rng.uniform(0.5 * nx, 2.0 * nx, size=nl - 1)
    phi = rng.uniform(0.0, 2 * np.pi, size=nl - 1)
    vel = np.sort(rng.uniform(V_MIN, V_MAX, size=nl))
    x = np.arange(nx)[None, :].astype(float)
    z = np.arange(nz)[:, None].astype(float)
    # fault: a line through (xf, 0) with dip angle; cells right of it are shifted by throw
    xf = rng.uniform(0.25 * nx, 0.75 * nx)
    dip = np.tan(rng.uniform(-0.6, 0.6))
    throw = rng.uniform(0.05 * nz, 0.2 * nz) * (1 if rng.random() < 0.5 else -1)
    side = (x - (xf + dip * z)) > 0
    zz = np.where(side, z - throw, z)
    layer = np.zeros((nz, nx), dtype=int)
    for i in range(nl - 1):
        iface = z0[i] + amp[i] * np.sin(2 * np.pi * x / lam[i] + phi[i])
        layer += (zz >= iface).astype(int)
    return vel[layer]


def linear_initial_model(nz: int = 70, nx: int = 70) -> np.ndarray:
    """1D linear gradient v(z) = 1500 + 3000 z/(nz-1), float64 [nz][nx]."""
    z = np.arange(nz, dtype=float)[:, None]
    return np.repeat(V_MIN + (V_MAX - V_MIN) * z / (nz - 1), nx, axis=1)


def model_batch(kind: str, seeds, nz: int = 70, nx: int = 70) -> np.ndarray:
    """Stack of models [B][nz][nx] (float64) for the given seeds."""
    gen = {"layered": layered_model, "curved_faulted": curved_faulted_model}[kind]
    return np.stack([gen(int(s), nz, nx) for s in seeds])


def smooth_perturbation(seed: int, nz: int, nx: int, scale: float) -> np.ndarray:
    """A smooth random field (sum of a few low-order sinusoids), max |.| = scale."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None] / max(nz - 1, 1)
    x = np.arange(nx)[None, :] / max(nx - 1, 1)
    f = np.zeros((nz, nx))
    for _ in range(4):
        kz, kx = rng.integers(1, 4, size=2)
        f += rng.normal() * np.sin(np.pi * kz * z + rng.uniform(0, 6.3)) * \
            np.sin(np.pi * kx * x + rng.uniform(0, 6.3))
    return scale * f / np.abs(f).max()


def gaussian_noise_like(d_clean: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """Additive Gaussian noise for Eq. (data_model) at a given SNR: per instance
    (leading axis) sigma^2 = mean(d_clean^2) / 10^(snr/10)."""
    rng = np.random.default_rng(seed)
    d = np.asarray(d_clean, dtype=np.float64)
    axes = tuple(range(1, d.ndim))
    power = np.mean(d * d, axis=axes, keepdims=True)
    sigma = np.sqrt(power / 10.0 ** (snr_db / 10.0))
    return sigma * rng.standard_normal(d.shape)


def random_field(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random float64 array (used for dot-product tests and guided-step inputs)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def blurred_model(v: np.ndarray, width: float) -> np.ndarray:
    """A model smoothed by a separable Gaussian of standard deviation `width`
    cells (edges replicated): the blurry estimates a reverse diffusion makes
    in its early, high-noise steps.  width <= 0 returns a copy."""
    v = np.asarray(v, dtype=np.float64)
    if width <= 0:
        return v.copy()
    r = int(np.ceil(3 * width))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / width) ** 2)
    k /= k.sum()
    p = np.pad(v, r, mode="edge")
    p = np.apply_along_axis(lambda a: np.convolve(a, k, mode="valid"), 0, p)
    return np.apply_along_axis(lambda a: np.convolve(a, k, mode="valid"), 1, p)


def surrogate_training_models(seed0: int, n: int, nz: int = 70, nx: int = 70) -> np.ndarray:
    """n seeded models [n][nz][nx] (float64) for fitting a forward surrogate:
    by index k = seed0 + i, k mod 4 = 0 layered, 1 curved/faulted, 2 a
    curved/faulted model blurred by 1-8 cells, 3 the linear gradient model
    plus a smooth perturbation of up to 600 m/s and white noise of up to
    150 m/s; every model clipped to [1500, 4500]."""
    out = np.empty((n, nz, nx))
    for i in range(n):
        k = seed0 + i
        rng = np.random.default_rng(1_000_003 * k + 17)
        kind = k % 4
        if kind == 0:
            v = layered_model(k, nz, nx, nlayers=int(rng.integers(3, 6)))
        elif kind == 1:
            v = curved_faulted_model(k, nz, nx)
        elif kind == 2:
            v = blurred_model(curved_faulted_model(k, nz, nx), rng.uniform(1.0, 8.0))
        else:
            v = linear_initial_model(nz, nx) + smooth_perturbation(k, nz, nx,
                                                                   rng.uniform(0.0, 600.0))
            v += rng.uniform(0.0, 150.0) * rng.standard_normal((nz, nx))
        out[i] = np.clip(v, V_MIN, V_MAX)
    return out
