"""Shared helpers for the test suite (inputs, tolerances, comparisons)."""
import numpy as np

from paper_2308_03972_gb300 import inputs

W_REST = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
U_RMS = 0.05 / np.sqrt(3.0)  # rms Mach 0.05 in lattice units

# FP64 path vs FP64 oracle: norm-relative max |f_gpu - f_oracle| / max |f|.
TOL_FP64 = 1e-12


def norm_rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def random_state(nx, ny, k, seed, spread=0.02):
    """Generic near-rest positive f [9][ny][nx][k] (non-equilibrium)."""
    return inputs.random_positive_f(nx, ny, k, seed, W_REST, spread)


def turbulent_state(oracle, nx, ny, k, seed, pert=0.1):
    """f = f^eq(1, u_m) of a random-phase ensemble (oracle's f^eq)."""
    u, v = inputs.ensemble_velocity(nx, ny, k, seed, U_RMS, pert)
    return oracle.set_equilibrium(np.ones_like(u), u, v)


def osse_observations(nx, ny, nobs_x, nobs_y, rng_seed, cycle, truth_u, truth_v, sigma):
    """Observed (u, v) at a uniform lattice: truth plus sigma * N(0, 1)."""
    ix, iy = inputs.uniform_obs_points(nx, ny, nobs_x, nobs_y)
    eu, ev = inputs.obs_noise(rng_seed, cycle, len(ix))
    return ix, iy, truth_u[iy, ix] + sigma * eu, truth_v[iy, ix] + sigma * ev
