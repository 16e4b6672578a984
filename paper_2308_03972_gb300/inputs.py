"""Seeded synthetic inputs for the LBM-LETKF observing-system simulation.

This module is shared by the CUDA path and the CPU oracle. It draws random
numbers and builds input arrays only; it holds none of the method's
arithmetic (no equilibrium, collision, observation operator or analysis).

Inputs follow the paper's experiment (arXiv 2308.03972, Section 4):
  * initial velocity fields: random-phase, divergence-free fields built from a
    streamfunction whose shell energy spectrum goes as E(k) ~ k^-3 for
    1 <= |k| <= N/4, scaled to a chosen rms speed (the paper starts all runs
    from uncorrelated random states, Section 4.3);
  * ensemble: an independent random centre field plus, per member, an
    independent field of the same spectrum at a fraction of the rms speed;
  * large-scale forcing F^i (Section 4.1): the curl of a scalar F_e summed
    over integer wavevectors in a shell with Gaussian coefficients, frozen in
    time and scaled to a chosen rms acceleration;
  * observation points on a uniform lattice of interval p (Section 4.3);
  * standard-normal observation-noise draws, one stream per (seed, cycle).
Lattice units throughout (dx = dt = 1).
"""
from __future__ import annotations

import numpy as np


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(x) for x in key])


def random_velocity(nx: int, ny: int, seed: int, u_rms: float, kmax: float | None = None,
                    slope: float = -3.0, stream: int = 0):
    """Divergence-free random-phase velocity (u, v), each [ny][nx], float64.

    The streamfunction has |psi_hat(k)| ~ |k|^((slope - 3)/2) so the shell
    spectrum E(k) ~ k^slope, for 1 <= |k| <= kmax (default min(nx, ny)/4).
    u = d psi / dy, v = -d psi / dx; rms of |u| is u_rms.
    """
    if kmax is None:
        kmax = min(nx, ny) / 4.0
    rng = _rng(seed, stream, 0x5EED)
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
    kk = np.sqrt(kx * kx + ky * ky)
    amp = np.zeros((ny, nx))
    band = (kk >= 1.0) & (kk <= kmax)
    amp[band] = kk[band] ** ((slope - 3.0) / 2.0)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(ny, nx))
    psi_hat = amp * np.exp(1j * phase)
    # u = dpsi/dy, v = -dpsi/dx (spectral derivatives); real part keeps a real field.
    two_pi = 2.0 * np.pi
    u = np.real(np.fft.ifft2(1j * (two_pi * ky / ny) * psi_hat))
    v = np.real(np.fft.ifft2(-1j * (two_pi * kx / nx) * psi_hat))
    rms = np.sqrt(np.mean(u * u + v * v))
    if rms > 0:
        u *= u_rms / rms
        v *= u_rms / rms
    return u, v


def ensemble_velocity(nx: int, ny: int, members: int, seed: int, u_rms: float, pert: float = 0.1):
    """Member velocities (u, v), each [ny][nx][members]: an independent centre
    field plus pert * (an independent field of the same spectrum and rms)."""
    uc, vc = random_velocity(nx, ny, seed, u_rms, stream=0)
    u = np.empty((ny, nx, members))
    v = np.empty((ny, nx, members))
    for m in range(members):
        up, vp = random_velocity(nx, ny, seed, u_rms, stream=1 + m)
        u[:, :, m] = uc + pert * up
        v[:, :, m] = vc + pert * vp
    return u, v


def forcing_field(nx: int, ny: int, seed: int, amp: float, kmin: float = 3.0, kmax: float = 4.0):
    """Frozen large-scale acceleration F^i = grad F_e x i_z, [2][ny][nx].

    F_e = sum over integer wavevectors k with kmin <= |k| <= kmax in one
    half-plane (k and -k give the same mode) of
    (r1 . k) cos(k . xi) + (r2 . k) sin(k . xi), r1, r2 standard-normal
    2-vectors, xi = 2 pi (x / nx, y / ny). The field is scaled to rms
    amplitude amp (this absorbs the paper's F_e0 and dx factor).
    """
    rng = _rng(seed, 0xF0C)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    fx = np.zeros((ny, nx))
    fy = np.zeros((ny, nx))
    kint = int(np.ceil(kmax))
    for ky in range(0, kint + 1):
        for kx in range(-kint, kint + 1):
            if ky == 0 and kx <= 0:
                continue  # half-plane
            kmag = np.hypot(kx, ky)
            if kmag < kmin or kmag > kmax:
                continue
            r1 = rng.standard_normal(2)
            r2 = rng.standard_normal(2)
            a = r1[0] * kx + r1[1] * ky
            b = r2[0] * kx + r2[1] * ky
            ph = 2.0 * np.pi * (kx * x / nx + ky * y / ny)
            # dF_e/dx and dF_e/dy of a cos(ph) + b sin(ph), ph = kx x' + ky y'.
            dfe = -a * np.sin(ph) + b * np.cos(ph)
            gx = kx * dfe
            gy = ky * dfe
            # F^i = grad F_e x i_z = (dF_e/dy, -dF_e/dx).
            fx += gy
            fy += -gx
    rms = np.sqrt(np.mean(fx * fx + fy * fy))
    if rms > 0:
        fx *= amp / rms
        fy *= amp / rms
    return np.ascontiguousarray(np.stack([fx, fy]))


def uniform_obs_points(nx: int, ny: int, nobs_x: int, nobs_y: int, offset: int = 0):
    """Observation points on a uniform lattice: (i * px + offset, j * py + offset)."""
    px = nx // nobs_x
    py = ny // nobs_y
    jj, ii = np.meshgrid(np.arange(nobs_y), np.arange(nobs_x), indexing="ij")
    ix = (ii.ravel() * px + offset) % nx
    iy = (jj.ravel() * py + offset) % ny
    return ix.astype(np.int32), iy.astype(np.int32)


def obs_noise(seed: int, cycle: int, npts: int):
    """Standard-normal draws (eps_u[npts], eps_v[npts]) for one analysis cycle."""
    z = _rng(seed, cycle, 0x0B5).standard_normal(2 * npts)
    return z[:npts].copy(), z[npts:].copy()


def random_positive_f(nx: int, ny: int, members: int, seed: int, base, spread: float = 0.02):
    """Generic positive arrays [9][ny][nx][members] for unit tests:
    base[alpha] * (1 + spread * uniform(-1, 1)), base supplied by the caller."""
    base = np.asarray(base, dtype=np.float64).reshape(9, 1, 1, 1)
    z = _rng(seed, 0xF).uniform(-1.0, 1.0, size=(9, ny, nx, members))
    return np.ascontiguousarray(base * (1.0 + spread * z))
