"""Reduced-precision local Gram matrices (letkf_set_products) in the
mixed-precision analysis: binary32, TF32 and BF16 products with binary32
accumulation for C = (k-1)/beta I + Yh^T Yh and b = Yh^T d-hat, the
eigensolve kept FP64-accurate. Each mode against the FP64 oracle, within a
bound set by the precision of its products, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, norm_rel, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS

# Norm-relative bound per mode. A Gram entry carries relative error ~u (unit
# roundoff of the products: 2^-24, 2^-11, 2^-8), so w-bar and W move by
# ~u times the condition of C (below ~30 here) and the state by that times
# |dX| / |f| (~1e-2); the bounds leave a factor of ~10 over the estimate and
# keep the binary32 storage floor (1e-6) for FP32.
BOUND = {"fp32": 1e-6, "tf32": 2e-4, "bf16": 2e-3}


def _case(nx, ny, k, nox, noy, seed):
    f = turbulent_state(oracle, nx, ny, k, seed=seed, pert=0.2)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f = oracle.lbm_run(f, force, TAU0, CS, MU, 5)
    ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
    rng = np.random.default_rng(seed)
    _, u, v = oracle.moments(f)
    yu = u.mean(2)[iy, ix] + SIGMA * rng.standard_normal(len(ix))
    yv = v.mean(2)[iy, ix] + SIGMA * rng.standard_normal(len(ix))
    return f, ix, iy, yu, yv


def _run(gpu, f, ix, iy, yu, yv, d_cut, mode):
    _, ny, nx, k = f.shape
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.set_products(mode)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        out = e.get_f()
        e.sync()
    return out


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (32, 32, 16, 8, 8, 6.0),    # K = 16 tile, p from 2 to ~60
    (32, 28, 32, 8, 7, 7.0),    # K = 32
    (32, 32, 64, 16, 16, 6.0),  # K = 64, p up to ~250 (ensemble space)
    (24, 24, 20, 6, 6, 9.0),    # k not a multiple of 16 (zero-padded tile)
])
def test_reduced_products_within_precision_bounds(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + k)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    base = _run(gpu, f, ix, iy, yu, yv, d_cut, gpu.LBM_PROD_FP64)
    errs = {}
    for name, mode in (("fp32", gpu.LBM_PROD_FP32), ("tf32", gpu.LBM_PROD_TF32),
                       ("bf16", gpu.LBM_PROD_BF16)):
        got = _run(gpu, f, ix, iy, yu, yv, d_cut, mode)
        errs[name] = norm_rel(got, ref)
        assert errs[name] <= BOUND[name], (name, errs)
        if mode != gpu.LBM_PROD_FP32:
            assert norm_rel(got, base) > 0.0, name  # the reduced pass ran
    assert norm_rel(base, ref) <= 1e-6
    # Coarser products give larger errors.
    assert errs["bf16"] > errs["tf32"] >= 0.1 * errs["fp32"]


def test_product_mode_arguments(gpu):
    f = turbulent_state(oracle, 8, 8, 4, seed=1)
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.set_products(gpu.LBM_PROD_TF32)
        assert err.value.code == gpu.LBM_EINVAL
        e.set_products(gpu.LBM_PROD_FP64)
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        with pytest.raises(gpu.LbmError):
            e.set_products(7)


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (32, 32, 16, 8, 8, 6.0),
    (32, 32, 64, 16, 16, 6.0),
    (24, 24, 20, 6, 6, 9.0),
    (16, 16, 128, 8, 8, 100.0),  # two row ranges per column, passes of 16 columns
])
def test_double_binary32_gram_matches_fp64_gram(gpu, nx, ny, k, nox, noy, d_cut):
    """LBM_PROD_DF32 (the mixed context's default): C and b to FP64-class
    accuracy on the binary32 units. The analysis equals the FP64-product one
    to the binary32 storage of the state, and the default is this mode."""
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=2 * nx + k)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    fp64 = _run(gpu, f, ix, iy, yu, yv, d_cut, gpu.LBM_PROD_FP64)
    df32 = _run(gpu, f, ix, iy, yu, yv, d_cut, gpu.LBM_PROD_DF32)
    assert norm_rel(df32, ref) <= 1e-6
    # A Gram entry within ~1e-14 of FP64 moves the stored state by at most a
    # few binary32 units of g = f - w (|g| < 0.05): ~1e-8 of max |f|.
    assert norm_rel(df32, fp64) <= 2e-8
    _, ny_, nx_, k_ = f.shape
    with gpu.Ensemble(nx_, ny_, k_, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        default = e.get_f()
        e.sync()
    assert np.array_equal(default, df32)


def test_double_binary32_mode_needs_a_mixed_context(gpu):
    f = turbulent_state(oracle, 8, 8, 4, seed=1)
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.set_products(gpu.LBM_PROD_DF32)
        assert err.value.code == gpu.LBM_EINVAL
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.set_products(gpu.LBM_PROD_DF32)
        with pytest.raises(gpu.LbmError):
            e.set_products(5)
