"""The hand-written CUDA adjoint of the LBM forecast (lbm_misfit,
lbm_misfit_gradient, and the torch.autograd.Function over them) against the
oracle gradient (float64 reverse-mode differentiation of the forecast), FP64
central finite differences of the misfit, and the FP64 adjoint for the
binary32 one, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as oracle_adjoint
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, norm_rel, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS


def _window_case(nx, ny, k, nsteps, every, side, seed):
    """Batch of k initial states, observations of a nature run with noise."""
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f0 = turbulent_state(oracle, nx, ny, k, seed=seed, pert=0.5)
    tu, tv = inputs.random_velocity(nx, ny, seed + 100, U_RMS)
    nat = oracle.set_equilibrium(np.ones((ny, nx, 1)), tu[:, :, None], tv[:, :, None])
    ix, iy = inputs.uniform_obs_points(nx, ny, side, side)
    yu, yv = [], []
    for t in range(1, nsteps + 1):
        nat = oracle.lbm_step(nat, force, TAU0, CS, MU)
        if t % every == 0:
            _, u, v = oracle.moments(nat)
            nu, nv = inputs.obs_noise(4, t, len(ix))
            yu.append(u[iy, ix, 0] + SIGMA * nu)
            yv.append(v[iy, ix, 0] + SIGMA * nv)
    return f0, force, {"nsteps": nsteps, "obs_every": every, "ix": ix, "iy": iy, "yo_u": np.array(yu),
                       "yo_v": np.array(yv), "sigma_u": SIGMA, "sigma_v": SIGMA}


def _win(gpu, w, checkpoint_every=20):
    return gpu.Window(w["nsteps"], w["obs_every"], w["ix"], w["iy"], w["yo_u"], w["yo_v"], w["sigma_u"],
                      w["sigma_v"], checkpoint_every=checkpoint_every)


@pytest.mark.parametrize("ckpt", [20, 7, 1, 100])
def test_fp64_gradient_matches_oracle_gradient_32x32(gpu, ckpt):
    nx = ny = 32
    k = 4
    f0, force, w = _window_case(nx, ny, k, 40, 10, 4, seed=5)
    weights = np.array([1.0, -0.5, 2.0, 0.25])
    Jr, gr, cr = oracle_adjoint.misfit_gradient(f0, force, TAU0, CS, MU, w, weights=weights)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0, force=force) as e:
        J, g, c = e.misfit_gradient(_win(gpu, w, ckpt), weights=weights)
        Jonly = e.misfit(_win(gpu, w, ckpt))
        after = e.get_f()
        e.sync()
    np.testing.assert_allclose(J, Jr, rtol=1e-12)
    np.testing.assert_allclose(Jonly, Jr, rtol=1e-12)
    assert norm_rel(g, gr) <= 1e-10
    np.testing.assert_allclose(c, cr, rtol=1e-9, atol=1e-12 * np.abs(cr).max())
    assert np.array_equal(after, f0)  # the context state is left as it was


def test_fp64_gradient_matches_central_differences(gpu):
    """16 random directions, h = 1e-6, on a 64^2 lattice of 8 states."""
    nx = ny = 64
    k = 8
    f0, force, w = _window_case(nx, ny, k, 60, 10, 8, seed=9)
    rng = np.random.default_rng(2)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0, force=force) as e:
        win = _win(gpu, w)
        J, g, c = e.misfit_gradient(win)
        h = 1e-6
        for _ in range(16):
            d = 1e-3 * rng.standard_normal(f0.shape)
            e.set_f(f0 + h * d)
            jp = e.misfit(win)
            e.set_f(f0 - h * d)
            jm = e.misfit(win)
            fd = (jp - jm) / (2 * h)
            ad = np.einsum("abcm,abcm->m", g, d)
            np.testing.assert_allclose(ad, fd, rtol=1e-5, atol=1e-12 * np.abs(J).max() / h)
        e.set_f(f0)
        e.set_closure(CS + h)
        jp = e.misfit(win)
        e.set_closure(CS - h)
        jm = e.misfit(win)
        e.sync()
    np.testing.assert_allclose(c, (jp - jm) / (2 * h), rtol=1e-5, atol=1e-12 * np.abs(J).max() / h)


def test_binary32_adjoint_close_to_fp64_adjoint(gpu):
    nx = ny = 64
    k = 8
    f0, force, w = _window_case(nx, ny, k, 60, 10, 8, seed=13)
    out = {}
    for prec in (gpu.LBM_FP64, gpu.LBM_MIXED):
        with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f0, force=force) as e:
            out[prec] = e.misfit_gradient(_win(gpu, w))
            e.sync()
    J64, g64, c64 = out[gpu.LBM_FP64]
    J32, g32, c32 = out[gpu.LBM_MIXED]
    np.testing.assert_allclose(J32, J64, rtol=1e-4)
    assert norm_rel(g32, g64) <= 1e-3
    np.testing.assert_allclose(c32, c64, rtol=1e-2)


def test_autograd_function_backward_is_the_adjoint(gpu):
    import torch

    from paper_2308_03972_gb300.adjoint import window_misfit

    nx = ny = 32
    k = 4
    f0, force, w = _window_case(nx, ny, k, 30, 10, 4, seed=21)
    upstream = np.array([0.5, 1.5, -1.0, 2.0])
    _, gr, cr = oracle_adjoint.misfit_gradient(f0, force, TAU0, CS, MU, w, weights=upstream)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, force=force) as e:
        x = torch.tensor(f0, device="cuda", requires_grad=True)
        cs = torch.tensor(CS, dtype=torch.float64, device="cuda", requires_grad=True)
        J = window_misfit(x, cs, e, _win(gpu, w))
        loss = (J * torch.tensor(upstream, device="cuda")).sum()
        gx, gc = torch.autograd.grad(loss, (x, cs))
        e.sync()
    assert norm_rel(gx.cpu().numpy(), gr) <= 1e-10
    assert abs(gc.item() / cr.sum() - 1) <= 1e-9


def test_window_argument_errors(gpu):
    f0 = turbulent_state(oracle, 8, 8, 2, seed=1)
    ix = np.array([1, 9], np.int32)
    with gpu.Ensemble(8, 8, 2, TAU0, CS, MU, gpu.LBM_FP64, f0=f0) as e:
        bad = gpu.Window(10, 5, ix, [1, 1], np.zeros((2, 2)), np.zeros((2, 2)), 0.1, 0.1)
        with pytest.raises(gpu.LbmError) as err:
            e.misfit(bad)
        assert err.value.code == gpu.LBM_EINVAL
        bad = gpu.Window(10, 5, [1, 1], [1, 1], np.zeros((2, 2)), np.zeros((2, 2)), 0.0, 0.1)
        with pytest.raises(gpu.LbmError):
            e.misfit_gradient(bad)
        bad = gpu.Window(0, 5, [1], [1], np.zeros((0, 1)), np.zeros((0, 1)), 0.1, 0.1)
        with pytest.raises(gpu.LbmError):
            e.misfit(bad)
        with pytest.raises(gpu.LbmError):
            e.set_closure(-0.1)


def test_adjoint_window_256x256_batch_64(gpu):
    """256^2 lattice, 64 initial states, 200-step window with (u, v) misfit
    at 16 x 16 points after every 10 steps, checkpoints every 20 steps: the
    FP64 adjoint against FP64 central differences (h = 1e-6, 16 random
    directions) and the binary32 adjoint against the FP64 one."""
    nx = ny = 256
    k = 64
    f0, force, w = _window_case(nx, ny, k, 200, 10, 16, seed=31)
    rng = np.random.default_rng(7)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0, force=force) as e:
        win = _win(gpu, w, 20)
        J64, g64, c64 = e.misfit_gradient(win)
        h = 1e-6
        for _ in range(16):
            d = 1e-3 * rng.standard_normal(f0.shape)
            e.set_f(f0 + h * d)
            jp = e.misfit(win)
            e.set_f(f0 - h * d)
            jm = e.misfit(win)
            ad = np.einsum("abcm,abcm->m", g64, d)
            np.testing.assert_allclose(ad, (jp - jm) / (2 * h), rtol=1e-5,
                                       atol=1e-12 * np.abs(J64).max() / h)
        e.sync()
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f0, force=force) as e:
        J32, g32, c32 = e.misfit_gradient(_win(gpu, w, 20))
        e.sync()
    np.testing.assert_allclose(J32, J64, rtol=1e-4)
    assert norm_rel(g32, g64) <= 1e-3
    np.testing.assert_allclose(c32, c64, rtol=1e-2)


def test_cs_gradient_sum_on_the_device(gpu):
    """dcs = sum_m w_m dJ_m/dC_s, summed on the device, host and device
    outputs, against the oracle's C_s derivative; device weights."""
    import torch

    nx = ny = 32
    k = 4
    f0, force, w = _window_case(nx, ny, k, 30, 10, 4, seed=9)
    weights = np.array([0.5, 1.0, -1.5, 2.0])
    _, _, cr = oracle_adjoint.misfit_gradient(f0, force, TAU0, CS, MU, w, weights=weights)
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0, force=force) as e:
        dh = np.zeros(1)
        _, gcs = gpu.lbm_misfit_gradient(e.ctx, _win(gpu, w), k, weights=weights, dcs=dh)
        wd = torch.tensor(weights, dtype=torch.float64, device="cuda")
        gd = torch.empty((9, ny, nx, k), dtype=torch.float64, device="cuda")
        dd = torch.zeros(1, dtype=torch.float64, device="cuda")
        gpu.lbm_misfit_gradient(e.ctx, _win(gpu, w), k, weights=wd, grad_f0=gd, dcs=dd)
        e.sync()
    total = float(np.sum(cr))
    assert abs(dh[0] - np.sum(gcs)) <= 1e-14 * np.abs(gcs).sum()
    assert abs(dh[0] - total) <= 1e-9 * abs(total) + 1e-12 * np.abs(cr).max()
    assert abs(float(dd.item()) - dh[0]) <= 1e-13 * abs(dh[0])  # per-block atomics: order varies
