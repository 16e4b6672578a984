"""Parity of the CUDA energy spectrum (lbm_energy_spectrum, Section 4.1 shell
spectrum, member mean as in Section 4.3) with the FP64 oracle, through the
C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7


def _spectrum_close(got, ref, rel=1e-12):
    """Every shell within rel of the largest shell energy."""
    return float(np.max(np.abs(got - ref)) / ref.max())


@pytest.mark.parametrize("nx,ny,k", [(48, 40, 8), (33, 31, 3), (64, 64, 1), (20, 36, 17)])
def test_spectrum_fp64_matches_oracle(gpu, nx, ny, k):
    f = turbulent_state(oracle, nx, ny, k, seed=nx + k, pert=0.3)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f = oracle.lbm_run(f, force, TAU0, CS, MU, 4)
    ref = oracle.energy_spectrum(f)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        got = e.energy_spectrum()
        e.sync()
    assert got.shape == ref.shape
    assert _spectrum_close(got, ref) <= 1e-12
    # Shells with non-negligible energy agree to relative rounding.
    big = ref > 1e-6 * ref.max()
    assert np.max(np.abs(got[big] / ref[big] - 1)) <= 1e-11


def test_spectrum_of_mixed_state_matches_oracle_of_that_state(gpu):
    nx, ny, k = 40, 32, 12
    f = turbulent_state(oracle, nx, ny, k, seed=7, pert=0.2)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.forecast(3)
        state = e.get_f()  # the binary32-stored state, widened to FP64
        got = e.energy_spectrum()
        e.sync()
    ref = oracle.energy_spectrum(state)
    assert _spectrum_close(got, ref) <= 1e-12


def test_spectrum_device_output_and_shell_counts(gpu):
    import torch

    nx, ny, k = 32, 24, 4
    f = turbulent_state(oracle, nx, ny, k, seed=11)
    nsh = gpu.spectrum_shells(nx, ny)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        host = e.energy_spectrum()
        dev = torch.full((nsh,), -1.0, dtype=torch.float64, device="cuda")
        e.energy_spectrum(dev)
        longer = e.energy_spectrum(np.full(nsh + 7, -1.0))
        shorter = e.energy_spectrum(np.full(5, -1.0))
        e.sync()
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)
    assert np.array_equal(longer[:nsh], host) and np.all(longer[nsh:] == 0.0)
    assert np.array_equal(shorter, host[:5])
    # Parseval: the shells hold the mean kinetic energy per unit mass.
    _, u, v = oracle.moments(f)
    assert abs(host.sum() / (0.5 * np.mean(u ** 2 + v ** 2)) - 1) <= 1e-12


def test_spectrum_rejects_bad_arguments(gpu):
    f = turbulent_state(oracle, 16, 16, 2, seed=1)
    with gpu.Ensemble(16, 16, 2, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.energy_spectrum(np.zeros(0))
        assert err.value.code == gpu.LBM_EINVAL


def test_single_mode_lands_in_its_shell(gpu):
    nx, ny = 64, 48
    A = 0.01
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    u = A * np.cos(2 * np.pi * (6 * x / nx + 8 * y / ny))
    with gpu.Ensemble(nx, ny, 1, TAU0, CS, MU, gpu.LBM_FP64) as e:
        e.set_equilibrium(None, u[:, :, None].copy(), np.zeros((ny, nx, 1)))
        E = e.energy_spectrum()
        e.sync()
    assert abs(E[10] - A * A / 4) <= 1e-13 * A * A
    assert np.max(np.abs(np.delete(E, 10))) <= 1e-14 * A * A


def test_velocity_rmse_on_the_device(gpu):
    """lbm_velocity_rmse against the RMSE of the two contexts' mean
    velocities (one member for the truth, several for the ensemble)."""
    nx, ny, k = 40, 24, 6
    u, v = inputs.ensemble_velocity(nx, ny, k, 7, U_RMS)
    tu, tv = inputs.random_velocity(nx, ny, 8, U_RMS)
    for prec in (gpu.LBM_FP64, gpu.LBM_MIXED):
        with gpu.Ensemble(nx, ny, k, 0.55, 0.2, 0.0, prec) as e, \
                gpu.Ensemble(nx, ny, 1, 0.55, 0.2, 0.0, gpu.LBM_FP64) as t:
            e.set_equilibrium(None, u, v)
            t.set_equilibrium(None, tu[:, :, None].copy(), tv[:, :, None].copy())
            e.forecast(3)
            t.forecast(3)
            r = e.velocity_rmse(t)
            um, vm = e.mean_velocity()
            ut, vt = t.mean_velocity()
            e.sync()
        ref = np.sqrt(np.mean((um - ut) ** 2 + (vm - vt) ** 2))
        assert abs(r / ref - 1) <= 1e-13
