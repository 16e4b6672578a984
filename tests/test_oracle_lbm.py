"""Pins of the oracle's lattice-Boltzmann step against what the paper and the
mathematics fix (arXiv 2308.03972, Section 2 and 4.1). CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
W_REST = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def _table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "d2q9.txt")) if l.strip() and not l.startswith("#")]
    cx = np.array([int(r[1]) for r in rows])
    cy = np.array([int(r[2]) for r in rows])
    w = np.array([int(r[3]) / int(r[4]) for r in rows])
    return cx, cy, w


def test_d2q9_table_matches_paper():
    cx, cy, w = oracle.d2q9()
    gx, gy, gw = _table()
    np.testing.assert_array_equal(cx, gx)
    np.testing.assert_array_equal(cy, gy)
    np.testing.assert_allclose(w, gw, rtol=0, atol=1e-17)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.02, -0.01), (0.97, -0.05, 0.04)])
def test_equilibrium_moments(rho, ux, uy):
    cx, cy, _ = _table()
    feq = oracle.equilibrium(rho, ux, uy)
    assert abs(feq.sum() - rho) < 1e-15
    assert abs((feq * cx).sum() - rho * ux) < 1e-16
    assert abs((feq * cy).sum() - rho * uy) < 1e-16
    # Second moment of the D2Q9 equilibrium: rho/3 I + rho u u.
    assert abs((feq * cx * cx).sum() - (rho / 3 + rho * ux * ux)) < 1e-15
    assert abs((feq * cx * cy).sum() - rho * ux * uy) < 1e-16
    assert abs((feq * cy * cy).sum() - (rho / 3 + rho * uy * uy)) < 1e-15


def _one_cell(f9, fix, fiy, tau0, cs, mu):
    """A 1x1 periodic lattice streams every population back to the same cell,
    so one step there is the collision alone."""
    f = np.asarray(f9, dtype=np.float64).reshape(9, 1, 1, 1)
    force = np.array([fix, fiy], dtype=np.float64).reshape(2, 1, 1)
    return oracle.lbm_step(f, force, tau0, cs, mu).reshape(9)


def test_collision_conserves_mass_and_adds_momentum():
    cx, cy, _ = _table()
    f = inputs.random_positive_f(1, 1, 6, seed=11, base=W_REST, spread=0.05)
    for m in range(6):
        f9 = f[:, 0, 0, m]
        fix, fiy, mu = 3e-4 * (m - 2), -2e-4 * m, 1e-3
        fs = _one_cell(f9, fix, fiy, 0.55, 0.2, mu)
        rho = f9.sum()
        ux, uy = (f9 * cx).sum() / rho, (f9 * cy).sum() / rho
        Fx, Fy = fix - mu * ux, fiy - mu * uy
        assert abs(fs.sum() - rho) < 1e-15
        assert abs((fs * cx).sum() - (rho * ux + rho * Fx)) < 1e-16
        assert abs((fs * cy).sum() - (rho * uy + rho * Fy)) < 1e-16


def test_forcing_term_moments_at_equilibrium():
    cx, cy, _ = _table()
    rho, ux, uy = 1.02, 0.03, -0.02
    feq = oracle.equilibrium(rho, ux, uy)
    fix, fiy, mu = 4e-4, -7e-4, 0.0
    Fa = _one_cell(feq, fix, fiy, 0.6, 0.2, mu) - feq
    # Fa is a difference of O(1) numbers: rounding is a few 1e-16.
    assert abs(Fa.sum()) < 1e-15
    assert abs((Fa * cx).sum() - rho * fix) < 1e-15
    assert abs((Fa * cy).sum() - rho * fiy) < 1e-15
    # First-order forcing: no second moment.
    assert abs((Fa * cx * cx).sum()) < 1e-15
    assert abs((Fa * cx * cy).sum()) < 1e-15


def test_smagorinsky_relaxation_time_solves_its_quadratic():
    cx, cy, _ = _table()
    f = inputs.random_positive_f(1, 1, 5, seed=12, base=W_REST, spread=0.1)
    tau0, cs = 0.55, 0.2
    for m in range(5):
        f9 = f[:, 0, 0, m]
        rho = f9.sum()
        ux, uy = (f9 * cx).sum() / rho, (f9 * cy).sum() / rho
        feq = oracle.equilibrium(rho, ux, uy)
        fs = _one_cell(f9, 0.0, 0.0, tau0, cs, 0.0)
        a = int(np.argmax(np.abs(f9 - feq)))
        tau = (f9[a] - feq[a]) / (f9[a] - fs[a])
        # Same relaxation time for every population.
        for b in range(9):
            np.testing.assert_allclose(f9[b] - fs[b], (f9[b] - feq[b]) / tau, rtol=0, atol=1e-15)
        neq = f9 - feq
        pxx, pxy, pyy = (cx * cx * neq).sum(), (cx * cy * neq).sum(), (cy * cy * neq).sum()
        Q = np.sqrt(2 * (pxx * pxx + 2 * pxy * pxy + pyy * pyy))
        # nu + nu_SGS = (tau - 1/2)/3 with nu_SGS = Cs^2 |S|, |S| = 3 Q / (2 rho tau):
        # tau^2 - tau0 tau - 9 Cs^2 Q / (2 rho) = 0.
        assert abs(tau * tau - tau0 * tau - 9 * cs * cs * Q / (2 * rho)) < 1e-12
        assert tau > tau0
        # Without the closure the relaxation time is tau0.
        fs0 = _one_cell(f9, 0.0, 0.0, tau0, 0.0, 0.0)
        np.testing.assert_allclose(f9 - fs0, (f9 - feq) / tau0, rtol=0, atol=1e-15)


def test_streaming_moves_each_population_along_its_velocity():
    cx, cy, _ = _table()
    nx, ny, k = 5, 4, 3
    f = inputs.random_positive_f(nx, ny, k, seed=13, base=W_REST, spread=0.05)
    force = inputs.forcing_field(nx, ny, seed=3, amp=1e-4, kmin=1, kmax=2)
    out = oracle.lbm_step(f, force, 0.55, 0.2, 1e-3)
    for y in range(ny):
        for x in range(nx):
            for m in range(k):
                fs = _one_cell(f[:, y, x, m], force[0, y, x], force[1, y, x], 0.55, 0.2, 1e-3)
                for a in range(9):
                    assert out[a, (y + cy[a]) % ny, (x + cx[a]) % nx, m] == fs[a]
    np.testing.assert_allclose(out.sum(), f.sum(), rtol=1e-15)


def test_uniform_force_accelerates_fluid_at_rest_exactly():
    nx, ny, k = 3, 3, 2
    rho = np.ones((ny, nx, k))
    z = np.zeros((ny, nx, k))
    f = oracle.set_equilibrium(rho, z, z)
    force = np.zeros((2, ny, nx))
    force[0] = 2e-5
    force[1] = -1e-5
    n = 25
    f = oracle.lbm_run(f, force, 0.55, 0.2, 0.0, n)
    r, u, v = oracle.moments(f)
    np.testing.assert_allclose(r, 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u, n * 2e-5, rtol=1e-11)
    np.testing.assert_allclose(v, -n * 1e-5, rtol=1e-11)


def test_linear_friction_decays_uniform_flow_geometrically():
    nx, ny, k = 2, 3, 1
    rho = np.ones((ny, nx, k))
    f = oracle.set_equilibrium(rho, np.full((ny, nx, k), 0.03), np.full((ny, nx, k), -0.01))
    mu, n = 2e-3, 40
    f = oracle.lbm_run(f, np.zeros((2, ny, nx)), 0.55, 0.2, mu, n)
    _, u, v = oracle.moments(f)
    np.testing.assert_allclose(u, 0.03 * (1 - mu) ** n, rtol=1e-12)
    np.testing.assert_allclose(v, -0.01 * (1 - mu) ** n, rtol=1e-12)


def _decay_rate(amps, t0, t1):
    return np.log(amps[t0] / amps[t1]) / (t1 - t0)


def test_shear_wave_decays_at_the_bgk_viscosity():
    """u_x = U sin(2 pi y / ny) decays as exp(-nu k^2 t), nu = (tau0 - 1/2)/3."""
    nx, ny, k = 4, 64, 1
    tau0 = 0.8
    y = np.arange(ny)
    u0 = 1e-3 * np.sin(2 * np.pi * y / ny)
    u = np.broadcast_to(u0[:, None, None], (ny, nx, k)).copy()
    f = oracle.set_equilibrium(np.ones((ny, nx, k)), u, np.zeros((ny, nx, k)))
    force = np.zeros((2, ny, nx))
    amps = {}
    for t in range(0, 1201):
        if t in (200, 1200):
            _, uu, _ = oracle.moments(f)
            amps[t] = 2 * np.mean(uu[:, 0, 0] * np.sin(2 * np.pi * y / ny))
        if t < 1200:
            f = oracle.lbm_step(f, force, tau0, 0.0, 0.0)
    nu = (tau0 - 0.5) / 3
    kk = 2 * np.pi / ny
    rate = _decay_rate(amps, 200, 1200)
    assert abs(rate / (nu * kk * kk) - 1) < 2e-3


def test_taylor_green_vortex_decay_and_smagorinsky_adds_dissipation():
    n, k = 32, 1
    tau0 = 0.55
    x = np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    kk = 2 * np.pi / n
    U = 2e-3
    u = (U * np.sin(kk * X) * np.cos(kk * Y))[:, :, None]
    v = (-U * np.cos(kk * X) * np.sin(kk * Y))[:, :, None]
    force = np.zeros((2, n, n))

    def energy_decay(cs):
        f = oracle.set_equilibrium(np.ones((n, n, k)), u, v)
        e = {}
        for t in range(0, 401):
            if t in (100, 400):
                _, uu, vv = oracle.moments(f)
                e[t] = np.mean(uu * uu + vv * vv)
            if t < 400:
                f = oracle.lbm_step(f, force, tau0, cs, 0.0)
        return _decay_rate(e, 100, 400)

    nu = (tau0 - 0.5) / 3
    rate0 = energy_decay(0.0)
    # Energy of the vortex decays as exp(-4 nu k^2 t) (amplitude exp(-2 nu k^2 t)).
    assert abs(rate0 / (4 * nu * kk * kk) - 1) < 1e-2
    assert energy_decay(0.2) > rate0 * (1 + 1e-4)


def test_observation_of_equilibrium_returns_velocity():
    ny, nx, k = 6, 5, 3
    rng = np.random.default_rng(5)
    rho = 1 + 0.01 * rng.standard_normal((ny, nx, k))
    u = 0.03 * rng.standard_normal((ny, nx, k))
    v = 0.03 * rng.standard_normal((ny, nx, k))
    f = oracle.set_equilibrium(rho, u, v)
    ix = np.array([0, 4, 2], np.int32)
    iy = np.array([5, 0, 3], np.int32)
    Y = oracle.observe(f, ix, iy)
    for j in range(3):
        np.testing.assert_allclose(Y[2 * j], u[iy[j], ix[j]], rtol=0, atol=1e-16)
        np.testing.assert_allclose(Y[2 * j + 1], v[iy[j], ix[j]], rtol=0, atol=1e-16)
    r2, u2, v2 = oracle.moments(f)
    np.testing.assert_allclose(r2, rho, rtol=1e-15)
    np.testing.assert_allclose(u2, u, rtol=0, atol=1e-16)


def _obs_fields(nox, noy, seed):
    rng = np.random.default_rng(seed)
    return (1 + 0.01 * rng.standard_normal((noy, nox)), 0.03 * rng.standard_normal((noy, nox)),
            0.03 * rng.standard_normal((noy, nox)))


def test_nudging_limits_and_moments():
    """Nudging (Section 3.1) is linear in gamma: gamma = 0 leaves f alone,
    gamma = 1 replaces it by f^eq of the interpolated observations, and the
    density moves as (1 - gamma) rho + gamma rho^."""
    nx, ny, k = 12, 8, 3
    f = inputs.random_positive_f(nx, ny, k, seed=21, base=W_REST, spread=0.05)
    ro, uo, vo = _obs_fields(4, 2, 1)
    np.testing.assert_array_equal(oracle.nudge(f, ro, uo, vo, 0.0), f)
    f1 = oracle.nudge(f, ro, uo, vo, 1.0)
    r1, u1, v1 = oracle.moments(f1)
    # At observation points the interpolation returns the observation itself.
    for j in range(2):
        for i in range(4):
            np.testing.assert_allclose(r1[j * 4, i * 3], ro[j, i], rtol=1e-14)
            np.testing.assert_allclose(u1[j * 4, i * 3], uo[j, i], rtol=0, atol=1e-15)
            np.testing.assert_allclose(v1[j * 4, i * 3], vo[j, i], rtol=0, atol=1e-15)
    # Halfway between two observation points in x: the mean of the two.
    np.testing.assert_allclose(u1[0, 1], (2 * uo[0, 0] + uo[0, 1]) / 3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(u1[4, 10], (2 * uo[1, 3] + uo[1, 0]) / 3, rtol=0, atol=1e-15)
    g = 0.3
    r0, _, _ = oracle.moments(f)
    rg, _, _ = oracle.moments(oracle.nudge(f, ro, uo, vo, g))
    np.testing.assert_allclose(rg, (1 - g) * r0 + g * r1, rtol=1e-14)


def test_dense_nudging_uses_the_observation_at_each_point():
    nx, ny, k = 6, 5, 2
    f = inputs.random_positive_f(nx, ny, k, seed=22, base=W_REST, spread=0.05)
    ro, uo, vo = _obs_fields(nx, ny, 2)
    r1, u1, v1 = oracle.moments(oracle.nudge(f, ro, uo, vo, 1.0))
    np.testing.assert_allclose(r1, np.broadcast_to(ro[:, :, None], r1.shape), rtol=1e-14)
    np.testing.assert_allclose(u1, np.broadcast_to(uo[:, :, None], u1.shape), rtol=0, atol=1e-15)
