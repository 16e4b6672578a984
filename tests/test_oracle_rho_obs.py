"""Oracle with the density observed as well as the velocity (Section 4.3
observes rho at the observation points with its own noise level), pinned to
facts other than itself: H returns the exact moments of an equilibrium
state; a density observation whose error is unbounded changes nothing; and,
because rho = sum_alpha f_alpha is linear in the state, a single density
observation updates the mean and variance of rho at its own cell by the
scalar Kalman formulas. CPU only."""
import numpy as np

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, turbulent_state


def test_observation_rows_are_u_v_rho():
    nx, ny, k = 12, 10, 3
    rng = np.random.default_rng(0)
    rho = 1.0 + 0.01 * rng.standard_normal((ny, nx, k))
    u = 0.02 * rng.standard_normal((ny, nx, k))
    v = 0.02 * rng.standard_normal((ny, nx, k))
    f = oracle.set_equilibrium(rho, u, v)
    ix = np.array([0, 5, 11], np.int32)
    iy = np.array([9, 3, 0], np.int32)
    Y = oracle.observe_vars(f, ix, iy, 3)
    for j in range(3):
        np.testing.assert_allclose(Y[3 * j], u[iy[j], ix[j]], rtol=0, atol=1e-15)
        np.testing.assert_allclose(Y[3 * j + 1], v[iy[j], ix[j]], rtol=0, atol=1e-15)
        np.testing.assert_allclose(Y[3 * j + 2], rho[iy[j], ix[j]], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(oracle.observe_vars(f, ix, iy, 2), oracle.observe(f, ix, iy))


def test_local_set_gives_three_scalars_per_point():
    ix = np.array([2, 9], np.int32)
    iy = np.array([2, 2], np.int32)
    idx, rl = oracle.local_obs_vars(16, 16, 2, 2, ix, iy, [0.1, 0.2, 0.05], 3.0)
    assert list(idx) == [0, 1, 2]  # the second point is 7 cells away (> 2 d_cut)
    np.testing.assert_allclose(rl, [1 / 0.01, 1 / 0.04, 1 / 0.0025], rtol=1e-15)


def _case(nx, ny, k, seed):
    f = turbulent_state(oracle, nx, ny, k, seed=seed, pert=0.3)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    return oracle.lbm_run(f, force, 0.55, 0.2, 6.16e-7, 4)


def test_unbounded_density_error_reduces_to_velocity_only():
    nx, ny, k = 16, 14, 6
    f = _case(nx, ny, k, 3)
    ix, iy = inputs.uniform_obs_points(nx, ny, 4, 2)
    rng = np.random.default_rng(1)
    yu = 0.01 * rng.standard_normal(len(ix))
    yv = 0.01 * rng.standard_normal(len(ix))
    yr = 1.0 + 0.001 * rng.standard_normal(len(ix))
    s = 0.1 * U_RMS
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, s, s, 5.0, 1.05)
    got = oracle.letkf_analyze_vars(f, ix, iy, np.stack([yu, yv, yr], 1), [s, s, 1e12], 5.0, 1.05)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_single_density_observation_is_the_scalar_kalman_update():
    nx, ny, k = 12, 12, 8
    f = _case(nx, ny, k, 5)
    ix = np.array([4], np.int32)
    iy = np.array([7], np.int32)
    rho_m = f[:, 7, 4, :].sum(axis=0)
    rbar = rho_m.mean()
    V = np.sum((rho_m - rbar) ** 2) / (k - 1)
    beta, sigma = 1.1, 2e-4
    yo_r = rbar + 3e-4
    huge = 1e10  # velocity observations carry no weight
    out = oracle.letkf_analyze_vars(f, ix, iy, [[0.0, 0.0, yo_r]], [huge, huge, sigma], 4.0, beta)
    ra = out[:, 7, 4, :].sum(axis=0)
    K = beta * V / (beta * V + sigma * sigma)
    assert abs(ra.mean() - (rbar + K * (yo_r - rbar))) <= 1e-14
    va = np.sum((ra - ra.mean()) ** 2) / (k - 1)
    assert abs(va / ((1 - K) * beta * V) - 1) <= 1e-9
