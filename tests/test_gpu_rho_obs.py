"""Parity of the CUDA analysis with density observed as well as velocity
(letkf_observe_rho; Section 4.3 observes rho with its own noise level)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import TOL_FP64, U_RMS, norm_rel, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS
SIGMA_RHO = 1e-3


def _case(nx, ny, k, nox, noy, seed):
    f = turbulent_state(oracle, nx, ny, k, seed=seed, pert=0.2)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f = oracle.lbm_run(f, force, TAU0, CS, MU, 5)
    ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
    rng = np.random.default_rng(seed)
    _, u, v = oracle.moments(f)
    yu = u.mean(2)[iy, ix] + SIGMA * rng.standard_normal(len(ix))
    yv = v.mean(2)[iy, ix] + SIGMA * rng.standard_normal(len(ix))
    yr = 1.0 + SIGMA_RHO * rng.standard_normal(len(ix))
    return f, ix, iy, yu, yv, yr


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (24, 20, 8, 4, 4, 6.0),    # p >= k: ensemble-space form
    (24, 24, 40, 4, 4, 5.0),   # p < k: observation-space form, p a multiple of 3
    (30, 26, 20, 3, 2, 9.5),   # ragged lattice, both forms across the grid
])
def test_analysis_with_density_fp64_matches_oracle(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv, yr = _case(nx, ny, k, nox, noy, seed=nx + k)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        e.observe_rho(ix, iy, yu, yv, yr, SIGMA, SIGMA, SIGMA_RHO)
        e.analyze(d_cut, 1.05)
        got = e.get_f()
        e.sync()
    ref = oracle.letkf_analyze_vars(f, ix, iy, np.stack([yu, yv, yr], 1), [SIGMA, SIGMA, SIGMA_RHO],
                                    d_cut, 1.05)
    assert norm_rel(got, ref) <= TOL_FP64
    # The density observations matter: velocity-only differs.
    uv = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    assert norm_rel(uv, ref) > 1e-9


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [(24, 20, 8, 4, 4, 6.0), (24, 24, 40, 4, 4, 5.0)])
def test_analysis_with_density_mixed_close_to_oracle(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv, yr = _case(nx, ny, k, nox, noy, seed=7 + k)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.observe_rho(ix, iy, yu, yv, yr, SIGMA, SIGMA, SIGMA_RHO)
        e.analyze(d_cut, 1.05)
        got = e.get_f()
        e.sync()
    ref = oracle.letkf_analyze_vars(f, ix, iy, np.stack([yu, yv, yr], 1), [SIGMA, SIGMA, SIGMA_RHO],
                                    d_cut, 1.05)
    assert norm_rel(got, ref) <= 1e-6


def test_switching_between_velocity_and_density_observations(gpu):
    """Consecutive analyses alternate the observation vector; buffers,
    geometry cache and local-problem sizing follow."""
    nx, ny, k = 20, 20, 12
    f, ix, iy, yu, yv, yr = _case(nx, ny, k, 4, 4, seed=31)
    sig3 = [SIGMA, SIGMA, SIGMA_RHO]
    ref = f
    ref = oracle.letkf_analyze(ref, ix, iy, yu, yv, SIGMA, SIGMA, 6.0, 1.05)
    ref = oracle.letkf_analyze_vars(ref, ix, iy, np.stack([yu, yv, yr], 1), sig3, 6.0, 1.05)
    ref = oracle.letkf_analyze(ref, ix[:5], iy[:5], yu[:5], yv[:5], SIGMA, SIGMA, 6.0, 1.05)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(6.0, 1.05)
        e.observe_rho(ix, iy, yu, yv, yr, *sig3)
        e.analyze(6.0, 1.05)
        e.observe(ix[:5], iy[:5], yu[:5], yv[:5], SIGMA, SIGMA)
        e.analyze(6.0, 1.05)
        got = e.get_f()
        e.sync()
    assert norm_rel(got, ref) <= TOL_FP64


def test_density_observation_argument_errors(gpu):
    f = turbulent_state(oracle, 8, 8, 4, seed=1)
    ix = np.array([1, 2], np.int32)
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        for bad in (0.0, -1.0, np.inf, np.nan):
            with pytest.raises(gpu.LbmError) as err:
                e.observe_rho(ix, ix, [0.0, 0.0], [0.0, 0.0], [1.0, 1.0], 0.1, 0.1, bad)
            assert err.value.code == gpu.LBM_EINVAL
        with pytest.raises(gpu.LbmError) as err:
            e.observe_rho(ix, ix, [0.0, 0.0], [0.0, 0.0], [1.0, np.nan], 0.1, 0.1, 0.01)
        assert err.value.code == gpu.LBM_EINVAL
