"""The reduced-precision Gram of the ensemble-space form (Section 3.2,
C = (k-1)/beta I + Yh^T Yh) on the tcgen05 tensor cores, TF32 and BF16
products with FP32 accumulation, against the FP64 oracle's analysis through
the C ABI. The cases cover every member tile (16, 32, 64, 128; points of a
block stacked two to eight to an MMA), members that are not a multiple of
four (rows staged by plain loads instead of TMA), ragged last stages of the
merged local set, lattices whose point count is not a multiple of the
block's eight points, and (u, v, rho) observations."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, norm_rel, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS
# Bounds of max |f^a - oracle| / max |f^a| (those of the 256^2 sweep).
BOUND = {"tf32": 2e-4, "bf16": 2e-3}


def _binary32_exact(f):
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4).reshape(9, 1, 1, 1)
    return (f - w).astype(np.float32).astype(np.float64) + w


# (nx, ny, k, obs lattice, d_cut): every case has ensemble-space points
# (p >= k) and n = min(k, p) <= 128.
CASES = [
    (48, 40, 16, 12, 10, 8.0),   # tile 16: eight points per MMA
    (44, 40, 18, 11, 10, 8.0),   # k = 18: plain-load staging, tile 32
    (40, 40, 32, 10, 10, 8.0),   # tile 32: four points per MMA
    (36, 36, 37, 12, 12, 7.0),   # k = 37: plain loads, tile 64
    (32, 36, 64, 16, 12, 6.0),   # tile 64: two points per MMA; 1152 points
    (30, 30, 128, 15, 15, 8.0),  # tile 128: two passes of four points; 900 points
]


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", CASES)
@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tensor_core_gram_matches_oracle(gpu, nx, ny, k, nox, noy, d_cut, mode):
    f = _binary32_exact(turbulent_state(oracle, nx, ny, k, seed=nx + k, pert=0.2))
    ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
    tu, tv = inputs.random_velocity(nx, ny, 400 + k, U_RMS)
    nu, nv = inputs.obs_noise(4, 1, len(ix))
    yu = tu[iy, ix] + SIGMA * nu
    yv = tv[iy, ix] + SIGMA * nv
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    prod = gpu.LBM_PROD_TF32 if mode == "tf32" else gpu.LBM_PROD_BF16
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.set_products(prod)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        got = e.get_f()
        e.sync()
    err = norm_rel(got, ref)
    assert err <= BOUND[mode], err
    # The reduced products do change the result: the path is the one
    # under test, not the FP64 Gram.
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        exact = e.get_f()
        e.sync()
    # FP64 Gram: binary32 storage and transform sums over up to 128 members.
    assert norm_rel(exact, ref) <= 2e-7
    assert np.max(np.abs(got - exact)) > 0.0


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tensor_core_gram_with_density_observations(gpu, mode):
    """(u, v, rho) at every point of the observation lattice: three rows per
    point in the merged local set."""
    nx, ny, k, no, d_cut = 40, 36, 32, 10, 7.0
    f = _binary32_exact(turbulent_state(oracle, nx, ny, k, seed=77, pert=0.2))
    ix, iy = inputs.uniform_obs_points(nx, ny, no, no)
    tu, tv = inputs.random_velocity(nx, ny, 500, U_RMS)
    nu, nv = inputs.obs_noise(4, 2, len(ix))
    nr, _ = inputs.obs_noise(5, 2, len(ix))
    yu = tu[iy, ix] + SIGMA * nu
    yv = tv[iy, ix] + SIGMA * nv
    srho = 1e-3
    yr = 1.0 + srho * nr
    ref = oracle.letkf_analyze_vars(f, ix, iy, np.stack([yu, yv, yr], 1), [SIGMA, SIGMA, srho], d_cut, 1.05)
    prod = gpu.LBM_PROD_TF32 if mode == "tf32" else gpu.LBM_PROD_BF16
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.set_products(prod)
        e.observe_rho(ix, iy, yu, yv, yr, SIGMA, SIGMA, srho)
        e.analyze(d_cut, 1.05)
        got = e.get_f()
        e.sync()
    assert norm_rel(got, ref) <= BOUND[mode]
