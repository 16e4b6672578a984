"""Oracle gradient of a windowed observation misfit through the LBM forecast.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the test
suite, the smoke check and the benchmark's CPU leg may import it.

The paper motivates its ensemble method by the cost of the adjoint model a
variational method needs (Section 1). This module gives the quantity such an
adjoint computes, for the forecast model of Section 2 / Section 4.1, in the
plainest form available: the forecast restated step by step in float64
PyTorch CPU tensors (the same readings as the C oracle ``lbm.c``: push
streaming, unforced f^eq in the non-equilibrium flux, F = F^i - mu u, no
force shift), the misfit

    J_m = 1/2 sum_{t in T} sum_j [ (u_m(eta_j, t) - yo_u[t, j])^2 / sigma_u^2
                                  + (v_m(eta_j, t) - yo_v[t, j])^2 / sigma_v^2 ],
    T = {e, 2e, ..., <= nsteps} (e = obs_every),

per member m, and its gradient by reverse-mode automatic differentiation
(``torch.autograd``) with respect to the initial f of each member and the
Smagorinsky coefficient C_s (one copy per member, so the gradient is per
member). Members are independent, so the gradient of sum_m w_m J_m with
respect to member m's f0 is w_m dJ_m/df0_m.
"""
from __future__ import annotations

import numpy as np
import torch

# D2Q9 in the order rest, +x, -x, +y, -y, (+,+), (-,-), (+,-), (-,+).
_CX = (0, 1, -1, 0, 0, 1, -1, 1, -1)
_CY = (0, 0, 0, 1, -1, 1, -1, -1, 1)
_W = (4.0 / 9,) + (1.0 / 9,) * 4 + (1.0 / 36,) * 4


def lbm_step(f, force, tau0, cs, mu):
    """One collide + push step. f [9][ny][nx][k] float64 tensor; force
    [2][ny][nx]; cs a scalar or a [k] tensor (per member)."""
    rho = f.sum(0)
    jx = sum(_CX[a] * f[a] for a in range(9))
    jy = sum(_CY[a] * f[a] for a in range(9))
    ux = jx / rho
    uy = jy / rho
    uu = ux * ux + uy * uy
    feq = torch.stack([_W[a] * rho * (1 + 3 * (_CX[a] * ux + _CY[a] * uy)
                                      + 4.5 * (_CX[a] * ux + _CY[a] * uy) ** 2 - 1.5 * uu)
                       for a in range(9)])
    neq = f - feq
    pxx = sum(_CX[a] * _CX[a] * neq[a] for a in range(9))
    pxy = sum(_CX[a] * _CY[a] * neq[a] for a in range(9))
    pyy = sum(_CY[a] * _CY[a] * neq[a] for a in range(9))
    x = 2 * (pxx * pxx + 2 * pxy * pxy + pyy * pyy)
    pos = x > 0
    q = torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))
    tau = 0.5 * (tau0 + torch.sqrt(tau0 * tau0 + 18 * cs * cs * q / rho))
    fx = force[0][:, :, None] - mu * ux
    fy = force[1][:, :, None] - mu * uy
    fstar = torch.stack([f[a] - neq[a] / tau + 3 * _W[a] * rho * (fx * _CX[a] + fy * _CY[a])
                         for a in range(9)])
    return torch.stack([torch.roll(fstar[a], shifts=(_CY[a], _CX[a]), dims=(0, 1)) for a in range(9)])


def velocity_at(f, ix, iy):
    """(u, v) [npts][k] of every member at the points."""
    g = f[:, iy, ix, :]
    rho = g.sum(0)
    u = sum(_CX[a] * g[a] for a in range(9)) / rho
    v = sum(_CY[a] * g[a] for a in range(9)) / rho
    return u, v


def _misfit_t(f0, cs, force, tau0, mu, window):
    ix = torch.as_tensor(np.asarray(window["ix"]), dtype=torch.long)
    iy = torch.as_tensor(np.asarray(window["iy"]), dtype=torch.long)
    yo_u = torch.as_tensor(np.asarray(window["yo_u"], dtype=np.float64))
    yo_v = torch.as_tensor(np.asarray(window["yo_v"], dtype=np.float64))
    su, sv = float(window["sigma_u"]), float(window["sigma_v"])
    e = int(window["obs_every"])
    f = f0
    J = torch.zeros(f0.shape[3], dtype=torch.float64)
    for t in range(1, int(window["nsteps"]) + 1):
        f = lbm_step(f, force, tau0, cs, mu)
        if t % e == 0:
            u, v = velocity_at(f, ix, iy)
            r = t // e - 1
            J = J + 0.5 * (((u - yo_u[r][:, None]) / su) ** 2 + ((v - yo_v[r][:, None]) / sv) ** 2).sum(0)
    return J


def misfit(f0, force, tau0, cs, mu, window):
    """J [k] of the window. f0 [9][ny][nx][k]; window: dict with nsteps,
    obs_every, ix, iy, yo_u, yo_v ([nsteps // obs_every][npts]), sigma_u,
    sigma_v."""
    with torch.no_grad():
        f0 = torch.as_tensor(np.asarray(f0, dtype=np.float64))
        k = f0.shape[3]
        cs_t = torch.full((k,), float(cs), dtype=torch.float64)
        return _misfit_t(f0, cs_t, torch.as_tensor(np.asarray(force, dtype=np.float64)), tau0, mu,
                         window).numpy()


def misfit_gradient(f0, force, tau0, cs, mu, window, weights=None):
    """(J [k], dF/df0 [9][ny][nx][k], dF/dC_s [k]) for F = sum_m w_m J_m,
    w = weights (ones by default)."""
    f0 = torch.tensor(np.asarray(f0, dtype=np.float64), requires_grad=True)
    k = f0.shape[3]
    cs_t = torch.full((k,), float(cs), dtype=torch.float64, requires_grad=True)
    w = torch.ones(k, dtype=torch.float64) if weights is None else torch.as_tensor(
        np.asarray(weights, dtype=np.float64))
    J = _misfit_t(f0, cs_t, torch.as_tensor(np.asarray(force, dtype=np.float64)), tau0, mu, window)
    gf, gc = torch.autograd.grad((w * J).sum(), (f0, cs_t))
    return J.detach().numpy(), gf.numpy(), gc.numpy()
