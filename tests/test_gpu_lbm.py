"""Parity of the CUDA lattice-Boltzmann path with the FP64 oracle
(arXiv 2308.03972, Section 2 and 4.1), called through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import TOL_FP64, norm_rel, random_state, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7


def _ens(b, f, force, prec, tau0=TAU0, cs=CS, mu=MU):
    _, ny, nx, k = f.shape
    return b.Ensemble(nx, ny, k, tau0, cs, mu, prec, f0=f, force=force)


@pytest.mark.parametrize("nx,ny,k", [(1, 1, 1), (5, 3, 2), (37, 29, 3), (33, 17, 8), (16, 16, 64), (7, 9, 5)])
def test_one_step_fp64_matches_oracle(gpu, nx, ny, k):
    f = random_state(nx, ny, k, seed=nx * 100 + k, spread=0.05)
    force = inputs.forcing_field(nx, ny, seed=3, amp=1e-4, kmin=1, kmax=2)
    with _ens(gpu, f, force, gpu.LBM_FP64) as e:
        e.forecast(1)
        got = e.get_f()
    ref = oracle.lbm_step(f, force, TAU0, CS, MU)
    assert norm_rel(got, ref) <= TOL_FP64


def test_many_steps_fp64_matches_oracle_turbulent(gpu):
    nx, ny, k = 48, 40, 4
    f = turbulent_state(oracle, nx, ny, k, seed=2)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    with _ens(gpu, f, force, gpu.LBM_FP64) as e:
        e.forecast(60)
        got = e.get_f()
    ref = oracle.lbm_run(f, force, TAU0, CS, MU, 60)
    assert norm_rel(got, ref) <= TOL_FP64


def test_moments_and_equilibrium_match_oracle(gpu):
    nx, ny, k = 19, 23, 6
    rng = np.random.default_rng(8)
    rho = 1 + 0.01 * rng.standard_normal((ny, nx, k))
    u = 0.03 * rng.standard_normal((ny, nx, k))
    v = 0.03 * rng.standard_normal((ny, nx, k))
    for prec, tol in ((gpu.LBM_FP64, 1e-15), (gpu.LBM_MIXED, 1e-7)):
        with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec) as e:
            e.set_equilibrium(rho, u, v)
            got = e.get_f()
            r2, u2, v2 = e.moments_host()
        ref = oracle.set_equilibrium(rho, u, v)
        assert norm_rel(got, ref) <= tol
        rr, ur, vr = oracle.moments(ref)
        assert np.max(np.abs(r2 - rr)) <= 10 * tol
        assert np.max(np.abs(u2 - ur)) <= 10 * tol
        assert np.max(np.abs(v2 - vr)) <= 10 * tol


def test_mixed_precision_steps_stay_close_to_oracle(gpu):
    nx, ny, k = 40, 36, 8
    f = turbulent_state(oracle, nx, ny, k, seed=5)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    with _ens(gpu, f, force, gpu.LBM_MIXED) as e:
        e.forecast(50)
        got = e.get_f()
        _, u, v = e.moments_host()
    ref = oracle.lbm_run(f, force, TAU0, CS, MU, 50)
    _, ur, vr = oracle.moments(ref)
    # binary32 storage of f - w keeps ~1e-9 absolute per step.
    assert norm_rel(got, ref) <= 1e-6
    urms = np.sqrt(np.mean(ur**2 + vr**2))
    assert np.sqrt(np.mean((u - ur) ** 2 + (v - vr) ** 2)) <= 1e-4 * urms


def test_full_size_step_matches_oracle(gpu):
    """256 x 256 lattice, 64 members, the launch shape the benchmark uses."""
    nx = ny = 256
    k = 64
    f = turbulent_state(oracle, nx, ny, k, seed=7)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    with _ens(gpu, f, force, gpu.LBM_FP64) as e:
        e.forecast(1)
        got = e.get_f()
    ref = oracle.lbm_step(f, force, TAU0, CS, MU)
    assert norm_rel(got, ref) <= TOL_FP64


def test_nonfinite_state_is_reported_as_divergence(gpu):
    nx, ny, k = 8, 8, 2
    f = random_state(nx, ny, k, seed=1)
    f[3, 2, 5, 1] = np.nan
    for prec in (gpu.LBM_FP64, gpu.LBM_MIXED):
        with _ens(gpu, f, None, prec) as e:
            e.forecast(2)
            with pytest.raises(gpu.LbmError) as err:
                e.sync()
            assert err.value.code == gpu.LBM_EDIVERGED
            # The flag is cleared once reported; the context stays usable.
            e.set_f(random_state(nx, ny, k, seed=2))
            e.forecast(1)
            e.sync()


def test_device_pointer_io_matches_host_io(gpu):
    import torch

    nx, ny, k = 12, 10, 4
    f = random_state(nx, ny, k, seed=4)
    with _ens(gpu, f, None, gpu.LBM_FP64) as e:
        e.forecast(3)
        host = e.get_f()
        dev = torch.empty((9, ny, nx, k), dtype=torch.float64, device="cuda")
        e.get_f(dev)
        u_d = torch.empty((ny, nx, k), dtype=torch.float64, device="cuda")
        e.moments(None, u_d, None)
        torch.cuda.synchronize()
        _, u_h, _ = e.moments_host()
    np.testing.assert_array_equal(dev.cpu().numpy(), host)
    np.testing.assert_array_equal(u_d.cpu().numpy(), u_h)


def test_mean_velocity_matches_oracle_moments(gpu):
    nx, ny, k = 21, 13, 7
    f = random_state(nx, ny, k, seed=6)
    for prec, tol in ((gpu.LBM_FP64, 1e-15), (gpu.LBM_MIXED, 1e-7)):
        with _ens(gpu, f, None, prec) as e:
            e.forecast(2)
            um, vm = e.mean_velocity()
        ref = oracle.lbm_run(f, np.zeros((2, ny, nx)), TAU0, CS, MU, 2)
        _, u, v = oracle.moments(ref)
        assert np.max(np.abs(um - u.mean(axis=2))) <= tol
        assert np.max(np.abs(vm - v.mean(axis=2))) <= tol
