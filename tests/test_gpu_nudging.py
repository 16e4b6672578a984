"""Parity of the CUDA nudging kernel (arXiv 2308.03972, Section 3.1) with
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from _helpers import TOL_FP64, norm_rel, random_state, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7


def _obs(nox, noy, seed):
    rng = np.random.default_rng(seed)
    return (1 + 0.01 * rng.standard_normal((noy, nox)), 0.03 * rng.standard_normal((noy, nox)),
            0.03 * rng.standard_normal((noy, nox)))


@pytest.mark.parametrize("nx,ny,k,nox,noy,gamma", [(24, 16, 8, 4, 4, 0.11), (30, 21, 3, 5, 7, 0.31),
                                                    (16, 16, 64, 16, 16, 0.2), (12, 12, 1, 3, 4, 1.0)])
def test_nudging_matches_oracle(gpu, nx, ny, k, nox, noy, gamma):
    f = random_state(nx, ny, k, seed=nx + k, spread=0.05)
    ro, uo, vo = _obs(nox, noy, 7)
    ref = oracle.nudge(f, ro, uo, vo, gamma)
    for prec, tol in ((gpu.LBM_FP64, TOL_FP64), (gpu.LBM_MIXED, 1e-6)):
        with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f) as e:
            e.nudge(ro, uo, vo, gamma)
            got = e.get_f()
            e.sync()
        assert norm_rel(got, ref) <= tol


def test_nudging_cycle_matches_oracle(gpu):
    """Forecast and nudge alternately, as in the paper's nudging OSSE."""
    nx = ny = 32
    k = 2
    f0 = turbulent_state(oracle, nx, ny, k, seed=4)
    force = np.zeros((2, ny, nx))
    ref = f0
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0, force=force) as e:
        for c in range(5):
            ro, uo, vo = _obs(8, 8, 100 + c)
            e.forecast(10)
            e.nudge(ro, uo, vo, 0.11)
            ref = oracle.nudge(oracle.lbm_run(ref, force, TAU0, CS, MU, 10), ro, uo, vo, 0.11)
        got = e.get_f()
    assert norm_rel(got, ref) <= TOL_FP64


def test_nudging_rejects_bad_arguments(gpu):
    with gpu.Ensemble(12, 12, 2, TAU0, CS, MU, gpu.LBM_FP64) as e:
        ro, uo, vo = _obs(5, 4, 1)
        with pytest.raises(gpu.LbmError):
            e.nudge(ro, uo, vo, 0.1)  # 12 is not a multiple of 5
        ro, uo, vo = _obs(4, 4, 1)
        with pytest.raises(gpu.LbmError):
            e.nudge(ro, uo, vo, 1.5)
        ro[0, 0] = np.nan
        with pytest.raises(gpu.LbmError):
            e.nudge(ro, uo, vo, 0.1)
