"""Pins of the oracle's eigensolver, Gaspari-Cohn weight and LETKF analysis
(arXiv 2308.03972, Section 3.2) against closed forms, brute force and the
explicit Kalman-gain form of the same estimator. CPU only."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- eigensolver
@pytest.mark.parametrize("n", [1, 2, 3, 8, 25, 64])
def test_sym_eig_matches_lapack_and_reconstructs(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T + 0.5 * np.eye(n)
    lam, Q = oracle.sym_eig(A)
    ref = np.linalg.eigvalsh(A)
    scale = np.abs(ref).max()
    assert np.abs(lam - ref).max() <= 1e-13 * scale
    assert np.abs(Q @ np.diag(lam) @ Q.T - A).max() <= 1e-13 * scale
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 1e-13


def test_sym_eig_indefinite_and_repeated_eigenvalues():
    rng = np.random.default_rng(7)
    n = 12
    Qr, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam_true = np.array([-3.0, -3.0, -1.0, 0.0, 0.0, 0.0, 2.0, 2.0, 5.0, 5.0, 5.0, 9.0])
    A = Qr @ np.diag(lam_true) @ Qr.T
    A = 0.5 * (A + A.T)
    lam, Q = oracle.sym_eig(A)
    assert np.abs(lam - lam_true).max() < 1e-13 * 9
    assert np.abs(Q @ np.diag(lam) @ Q.T - A).max() < 1e-13 * 9
    lam, Q = oracle.sym_eig(np.eye(5) * 2.5)
    np.testing.assert_array_equal(lam, 2.5)


def test_sym_eig_tridiagonal_closed_form():
    # Eigenvalues of the n x n second-difference matrix: 2 - 2 cos(j pi / (n+1)).
    n = 20
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    lam, _ = oracle.sym_eig(A)
    ref = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    assert np.abs(lam - ref).max() < 1e-14


# --------------------------------------------------------------- Gaspari-Cohn
def test_gaspari_cohn_exact_values_from_printed_formula():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gaspari_cohn.txt")) if l.strip() and not l.startswith("#")]
    for d, num, den in rows:
        assert abs(oracle.gaspari_cohn(float(d)) - int(num) / int(den)) < 1e-15


def test_gaspari_cohn_is_continuous_smooth_and_near_gaussian():
    G = oracle.gaspari_cohn
    h = 1e-6
    # Both branches meet at d = 1 with the same value and slope.
    assert abs(G(1 - 1e-12) - G(1 + 1e-12)) < 1e-11
    slope_lo = (G(1.0) - G(1.0 - h)) / h
    slope_hi = (G(1.0 + h) - G(1.0)) / h
    assert abs(slope_lo - slope_hi) < 1e-5
    # Compact support: value and slope vanish at d = 2.
    assert abs(G(2 - 1e-9)) < 1e-15
    assert abs((G(2.0) - G(2.0 - h)) / h) < 1e-9
    assert G(2.0) == 0.0 and G(3.7) == 0.0
    # Close to exp(-1.5 d^2) on [0, 2] and monotone decreasing.
    ds = np.linspace(0, 2, 401)
    g = np.array([G(d) for d in ds])
    assert np.abs(g - np.exp(-1.5 * ds * ds)).max() < 0.03
    assert np.all(np.diff(g) <= 0)


# ------------------------------------------------------------- LETKF algebra
def _ensemble_problem(n, k, p, seed, beta=1.0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k)) + 3.0
    H = rng.standard_normal((p, n))
    sig = 0.3 + rng.uniform(0, 1, p)
    y = rng.standard_normal(p)
    return X, H, sig, y


@pytest.mark.parametrize("k,n,p,beta", [(3, 5, 2, 1.0), (4, 10, 3, 1.05), (8, 30, 10, 1.2), (8, 6, 1, 1.0)])
def test_unlocalised_etkf_equals_kalman_gain(k, n, p, beta):
    """With linear H and no localisation, the ETKF mean is the Kalman update
    x + K (y - H x) and its sample covariance is (I - K H) P^b, with
    P^b = beta dX dX^T / (k - 1) and K = P^b H^T (H P^b H^T + R)^-1."""
    X, H, sig, y = _ensemble_problem(n, k, p, seed=100 * k + p, beta=beta)
    xbar = X.mean(axis=1)
    dX = X - xbar[:, None]
    Y = H @ X
    dY = Y - Y.mean(axis=1, keepdims=True)
    d = y - Y.mean(axis=1)
    Xa = oracle.letkf_update(X, dY, 1.0 / sig**2, d, beta)
    Pb = beta * dX @ dX.T / (k - 1)
    R = np.diag(sig**2)
    K = Pb @ H.T @ np.linalg.solve(H @ Pb @ H.T + R, np.eye(p))
    mean_ref = xbar + K @ (y - H @ xbar)
    cov_ref = (np.eye(n) - K @ H) @ Pb
    xa_bar = Xa.mean(axis=1)
    dXa = Xa - xa_bar[:, None]
    cov = dXa @ dXa.T / (k - 1)
    assert np.abs(xa_bar - mean_ref).max() < 1e-12 * np.abs(mean_ref).max()
    assert np.abs(cov - cov_ref).max() < 1e-12 * np.abs(Pb).max()


def test_localisation_weights_act_as_scaled_error_variances():
    """R-localisation R_loc^-1 = G o R^-1: the update with weights g equals the
    Kalman update with observation variances sigma^2 / g."""
    k, n, p = 6, 8, 5
    X, H, sig, y = _ensemble_problem(n, k, p, seed=42)
    g = np.array([1.0, 0.7, 0.3, 0.05, 0.9])
    xbar = X.mean(axis=1)
    dX = X - xbar[:, None]
    Y = H @ X
    dY = Y - Y.mean(axis=1, keepdims=True)
    Xa = oracle.letkf_update(X, dY, g / sig**2, y - Y.mean(axis=1), 1.0)
    Pb = dX @ dX.T / (k - 1)
    K = Pb @ H.T @ np.linalg.inv(H @ Pb @ H.T + np.diag(sig**2 / g))
    np.testing.assert_allclose(Xa.mean(axis=1), xbar + K @ (y - H @ xbar), rtol=1e-12)


def test_transform_structure():
    """W is symmetric positive definite, W 1 = sqrt(beta) 1 and 1^T wbar = 0,
    because dY 1 = 0 makes 1 an eigenvector of P-tilde."""
    rng = np.random.default_rng(3)
    k, p, beta = 10, 7, 1.05
    Yf = rng.standard_normal((p, k))
    dY = Yf - Yf.mean(axis=1, keepdims=True)
    rloc = rng.uniform(0.1, 2.0, p)
    d = rng.standard_normal(p)
    wbar, W = oracle.letkf_transform(dY, rloc, d, beta)
    assert np.abs(W - W.T).max() < 1e-14
    assert np.linalg.eigvalsh(0.5 * (W + W.T)).min() > 0
    np.testing.assert_allclose(W @ np.ones(k), np.sqrt(beta), rtol=1e-13)
    assert abs(wbar.sum()) < 1e-13
    # W^2 = (k - 1) P-tilde.
    C = (k - 1) / beta * np.eye(k) + dY.T @ np.diag(rloc) @ dY
    np.testing.assert_allclose(W @ W, (k - 1) * np.linalg.inv(C), rtol=0, atol=1e-13)


def test_no_observation_gives_pure_inflation():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((9, 5))
    xbar = X.mean(axis=1, keepdims=True)
    for beta in (1.0, 1.05):
        Xa = oracle.letkf_update(X, np.zeros((0, 5)), np.zeros(0), np.zeros(0), beta)
        np.testing.assert_allclose(Xa, xbar + np.sqrt(beta) * (X - xbar), rtol=0, atol=1e-14)


# ------------------------------------------------------- local observation set
def test_local_observation_set_brute_force():
    nx = ny = 256
    obs = [(i * 32, j * 32) for j in range(8) for i in range(8)]
    ix = np.array([o[0] for o in obs], np.int32)
    iy = np.array([o[1] for o in obs], np.int32)
    d_cut = 32.0
    counts = []
    for (x, y) in [(0, 0), (16, 16), (255, 3), (100, 200), (31, 0), (64, 128)]:
        idx, rl = oracle.local_obs(nx, ny, x, y, ix, iy, 0.1, 0.2, d_cut)
        exp = []
        for j, (ox, oy) in enumerate(obs):
            dx = min(abs(ox - x), nx - abs(ox - x))
            dy = min(abs(oy - y), ny - abs(oy - y))
            r = np.hypot(dx, dy)
            if r < 2 * d_cut:
                exp += [2 * j, 2 * j + 1]
        assert sorted(idx.tolist()) == exp
        g = np.array([oracle.gaspari_cohn(np.hypot(min(abs(ix[i // 2] - x), nx - abs(ix[i // 2] - x)),
                                                   min(abs(iy[i // 2] - y), ny - abs(iy[i // 2] - y))) / d_cut)
                      for i in idx])
        np.testing.assert_allclose(rl, g / np.where(idx % 2 == 0, 0.1**2, 0.2**2), rtol=1e-15)
        counts.append(len(idx))
    # On an observation point, the 3 x 3 block of neighbours is in range: 9 points, 18 scalars.
    assert counts[0] == 18


def test_analysis_of_grid_matches_pointwise_update():
    """letkf_analyze gathers H(x), dY, d and the local set, then applies the
    same transform as letkf_update at every point."""
    nx, ny, k = 12, 10, 5
    rng = np.random.default_rng(9)
    rho = 1 + 0.01 * rng.standard_normal((ny, nx, k))
    u = 0.02 * rng.standard_normal((ny, nx, k))
    v = 0.02 * rng.standard_normal((ny, nx, k))
    f = oracle.set_equilibrium(rho, u, v)
    f += 1e-4 * rng.standard_normal(f.shape)
    ix = np.array([0, 4, 8, 2, 9], np.int32)
    iy = np.array([0, 3, 7, 8, 1], np.int32)
    yo_u = 0.02 * rng.standard_normal(5)
    yo_v = 0.02 * rng.standard_normal(5)
    su, sv, d_cut, beta = 0.01, 0.015, 3.0, 1.05
    fa = oracle.letkf_analyze(f, ix, iy, yo_u, yo_v, su, sv, d_cut, beta)
    Y = oracle.observe(f, ix, iy)
    ybar = Y.mean(axis=1)
    dYall = Y - ybar[:, None]
    yo = np.empty(10)
    yo[0::2], yo[1::2] = yo_u, yo_v
    for (x, y) in [(0, 0), (5, 5), (11, 9), (3, 7)]:
        idx, rl = oracle.local_obs(nx, ny, x, y, ix, iy, su, sv, d_cut)
        Xa = oracle.letkf_update(f[:, y, x, :], dYall[idx], rl, (yo - ybar)[idx], beta)
        np.testing.assert_array_equal(fa[:, y, x, :], Xa)
    # A subset analysis touches only the listed cells.
    pts = np.array([3 * nx + 4, 7], np.int32)
    fs = oracle.letkf_analyze(f, ix, iy, yo_u, yo_v, su, sv, d_cut, beta, points=pts)
    mask = np.zeros((ny, nx), bool)
    mask.flat[pts] = True
    np.testing.assert_array_equal(fs[:, mask], fa[:, mask])
    np.testing.assert_array_equal(fs[:, ~mask], f[:, ~mask])
