"""Oracle energy spectrum (Section 4.1) pinned to facts other than itself:
single Fourier modes land in the shell of their magnitude with the energy
the definition gives in closed form; Parseval's identity; the member mean;
a numpy FFT of the same velocity field (a library routine of the same
definition). CPU only."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS


def _state_from_velocity(u, v):
    """f^eq(1, u, v) for fields [ny][nx][k]; its moments return u, v."""
    return oracle.set_equilibrium(np.ones_like(u), u, v)


@pytest.mark.parametrize("nx,ny,kx,ky", [(32, 32, 3, 4), (48, 40, 1, 1), (40, 48, 5, 0), (33, 31, 2, 7)])
def test_single_mode_energy_in_its_shell(nx, ny, kx, ky):
    # u = A cos(2 pi (kx x / nx + ky y / ny)): u-hat = A/2 at +-(kx, ky), so
    # E = 2 * (A/2)^2 / 2 = A^2 / 4, all in shell round(|(kx, ky)|).
    A = 0.01
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    u = A * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny))
    f = _state_from_velocity(u[:, :, None], np.zeros((ny, nx, 1)))
    E = oracle.energy_spectrum(f)
    s = int(np.floor(np.hypot(kx, ky) + 0.5))
    assert abs(E[s] - A * A / 4) <= 1e-13 * A * A
    rest = np.delete(E, s)
    assert np.max(np.abs(rest)) <= 1e-14 * A * A


def test_constant_flow_is_shell_zero():
    nx, ny = 16, 12
    u = np.full((ny, nx, 2), 0.02)
    v = np.full((ny, nx, 2), -0.01)
    E = oracle.energy_spectrum(_state_from_velocity(u, v))
    assert abs(E[0] - 0.5 * (0.02 ** 2 + 0.01 ** 2)) <= 1e-16
    assert np.max(np.abs(E[1:])) <= 1e-18


def test_parseval_and_member_mean():
    nx, ny, k = 40, 36, 3
    u, v = inputs.ensemble_velocity(nx, ny, k, 5, U_RMS, 0.3)
    f = _state_from_velocity(u, v)
    E = oracle.energy_spectrum(f)
    # Parseval with u-hat = N^{-1} sum: sum_k' E(k') = <|u|^2> / 2 per member.
    want = 0.5 * np.mean(u ** 2 + v ** 2)
    assert abs(E.sum() - want) <= 1e-13 * want
    per_member = [oracle.energy_spectrum(f[..., m:m + 1]) for m in range(k)]
    assert np.max(np.abs(E - np.mean(per_member, axis=0))) <= 1e-15 * E.max()


def test_matches_numpy_fft_shell_sums():
    nx, ny, k = 24, 20, 2
    u, v = inputs.ensemble_velocity(nx, ny, k, 9, U_RMS, 0.5)
    f = _state_from_velocity(u, v)
    _, um, vm = oracle.moments(f)
    nsh = oracle.spectrum_shells(nx, ny)
    want = np.zeros(nsh)
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
    shell = np.floor(np.hypot(kx, ky) + 0.5).astype(int)
    for m in range(k):
        e = 0.5 * (np.abs(np.fft.fft2(um[:, :, m]) / (nx * ny)) ** 2 +
                   np.abs(np.fft.fft2(vm[:, :, m]) / (nx * ny)) ** 2)
        want += np.bincount(shell.ravel(), weights=e.ravel(), minlength=nsh)[:nsh] / k
    got = oracle.energy_spectrum(f)
    assert np.max(np.abs(got - want)) <= 1e-13 * want.max()


def test_truncated_shell_count_drops_high_shells():
    nx, ny, k = 16, 16, 1
    u, v = inputs.ensemble_velocity(nx, ny, k, 2, U_RMS, 0.0)
    f = _state_from_velocity(u, v)
    full = oracle.energy_spectrum(f)
    part = oracle.energy_spectrum(f, 5)
    assert np.array_equal(part, full[:5])
