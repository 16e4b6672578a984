"""The oracle gradient of the windowed misfit (oracle/adjoint.py) pinned to
facts other than itself: its float64 forecast equals the C oracle's step by
step, and its gradient equals central finite differences of the misfit
computed with the C oracle's forecast, for the initial state (random
directions) and for the Smagorinsky coefficient. CPU only."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, turbulent_state

TAU0, MU = 0.55, 6.16e-7


def _setup(nx, ny, k, seed, nsteps, every, npts_side):
    f0 = turbulent_state(oracle, nx, ny, k, seed=seed, pert=0.3)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f0 = oracle.lbm_run(f0, force, TAU0, 0.2, MU, 2)  # away from equilibrium
    ix, iy = inputs.uniform_obs_points(nx, ny, npts_side, npts_side)
    rng = np.random.default_rng(seed)
    nt = nsteps // every
    sigma = 0.1 * U_RMS
    window = {"nsteps": nsteps, "obs_every": every, "ix": ix, "iy": iy,
              "yo_u": U_RMS * rng.standard_normal((nt, len(ix))),
              "yo_v": U_RMS * rng.standard_normal((nt, len(ix))), "sigma_u": sigma, "sigma_v": 1.5 * sigma}
    return f0, force, window


def _misfit_c(f0, force, cs, window):
    """J [k] from the C oracle's forecast and moments (independent code)."""
    f = f0
    J = np.zeros(f0.shape[3])
    ix, iy = window["ix"], window["iy"]
    for t in range(1, window["nsteps"] + 1):
        f = oracle.lbm_step(f, force, TAU0, cs, MU)
        if t % window["obs_every"] == 0:
            _, u, v = oracle.moments(f)
            r = t // window["obs_every"] - 1
            J += 0.5 * (((u[iy, ix] - window["yo_u"][r][:, None]) / window["sigma_u"]) ** 2 +
                        ((v[iy, ix] - window["yo_v"][r][:, None]) / window["sigma_v"]) ** 2).sum(0)
    return J


def test_forecast_equals_c_oracle():
    nx, ny, k = 12, 10, 3
    f, force, _ = _setup(nx, ny, k, 1, 4, 2, 2)
    ft = torch.as_tensor(f)
    fo = torch.as_tensor(force)
    for _ in range(5):
        ref = oracle.lbm_step(f, force, TAU0, 0.2, MU)
        ft = adjoint.lbm_step(ft, fo, TAU0, 0.2, MU)
        f = ref
        assert np.max(np.abs(ft.numpy() - ref)) <= 1e-15 * np.max(np.abs(ref))


def test_misfit_equals_c_oracle_misfit():
    f0, force, window = _setup(10, 12, 2, 4, 12, 4, 2)
    got = adjoint.misfit(f0, force, TAU0, 0.2, MU, window)
    ref = _misfit_c(f0, force, 0.2, window)
    assert np.max(np.abs(got / ref - 1)) <= 1e-12


@pytest.mark.parametrize("cs", [0.2, 0.0])
def test_gradient_matches_central_differences(cs):
    nx, ny, k = 10, 8, 2
    f0, force, window = _setup(nx, ny, k, 7, 15, 5, 2)
    J, gf, gc = adjoint.misfit_gradient(f0, force, TAU0, cs, MU, window)
    np.testing.assert_allclose(J, _misfit_c(f0, force, cs, window), rtol=1e-12)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(f0.shape) * 1e-2
        fd = (_misfit_c(f0 + h * d, force, cs, window) - _misfit_c(f0 - h * d, force, cs, window)) / (2 * h)
        ad = np.einsum("abcm,abcm->m", gf, d)
        np.testing.assert_allclose(ad, fd, rtol=2e-6, atol=1e-9 * np.abs(J).max())
    if cs > 0:
        fd = (_misfit_c(f0, force, cs + h, window) - _misfit_c(f0, force, cs - h, window)) / (2 * h)
        np.testing.assert_allclose(gc, fd, rtol=2e-6, atol=1e-9 * np.abs(J).max())


def test_member_weights_scale_member_gradients():
    f0, force, window = _setup(8, 8, 3, 2, 6, 3, 2)
    _, g1, c1 = adjoint.misfit_gradient(f0, force, TAU0, 0.2, MU, window)
    w = np.array([2.0, -0.5, 0.0])
    _, gw, cw = adjoint.misfit_gradient(f0, force, TAU0, 0.2, MU, window, weights=w)
    np.testing.assert_allclose(gw, g1 * w, rtol=1e-13, atol=0)
    np.testing.assert_allclose(cw, c1 * w, rtol=1e-13, atol=0)
