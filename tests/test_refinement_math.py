"""The matrix-function identities the CUDA analysis relies on, checked in
numpy against direct eigendecomposition (CPU only):

* the observation-space form of the LETKF transform (p < k): with
  Yh = diag(sqrt(rho)) dY, A = Yh Yh^T and a = (k-1)/beta,
  w-bar = Yh^T (aI + A)^{-1} d-hat and
  C^{-1/2} = a^{-1/2} I + Yh^T g(A) Yh, g(s) = ((a+s)^{-1/2} - a^{-1/2}) / s;
* the closed-form divided differences used to evaluate f(S) to first order
  in the off-diagonal of a nearly diagonal S (Daleckii-Krein);
* the refinement of a binary32 eigenbasis in FP64 (Rayleigh-Ritz, with the
  basis' non-orthogonality E = X^T X - I taken to first order instead of
  re-orthonormalising, first-order matrix functions): error O(|E|^2).
"""
import numpy as np
import pytest


def _problem(k, p, seed, beta=1.05):
    rng = np.random.default_rng(seed)
    Yf = 0.003 * rng.standard_normal((p, k))
    dY = Yf - Yf.mean(axis=1, keepdims=True)
    rho = rng.uniform(0.01, 1.0, p) / 0.00289**2
    d = 0.003 * rng.standard_normal(p)
    return dY, rho, d, (k - 1) / beta


def _fun(M, f):
    w, V = np.linalg.eigh(M)
    return V @ np.diag(f(w)) @ V.T


def test_observation_space_form_equals_ensemble_space_form():
    k, p = 64, 25
    dY, rho, d, a = _problem(k, p, 1)
    Yh = np.sqrt(rho)[:, None] * dY
    C = a * np.eye(k) + Yh.T @ Yh
    Pt = np.linalg.inv(C)
    wbar = Pt @ Yh.T @ (np.sqrt(rho) * d)
    Cih = _fun(C, lambda x: x ** -0.5)
    A = Yh @ Yh.T
    g = lambda s: ((a + s) ** -0.5 - a ** -0.5) / s  # noqa: E731
    wbar_obs = Yh.T @ np.linalg.solve(a * np.eye(p) + A, np.sqrt(rho) * d)
    Cih_obs = a ** -0.5 * np.eye(k) + Yh.T @ _fun(A, g) @ Yh
    np.testing.assert_allclose(wbar_obs, wbar, rtol=1e-12, atol=1e-14 * np.abs(wbar).max())
    np.testing.assert_allclose(Cih_obs, Cih, rtol=0, atol=1e-13 * np.abs(Cih).max())


@pytest.mark.parametrize("x,y", [(3.0, 7.0), (100.0, 100.0 + 1e-9), (0.5, 900.0), (0.0, 1e-12)])
def test_closed_form_divided_differences(x, y):
    a = 60.0
    r, u, w = np.sqrt(a), np.sqrt(a + x), np.sqrt(a + y)
    # g(s) = q[s, 0], q(s) = (a+s)^{-1/2}; g[x, y] in closed form.
    gxy = (u + w + r) / (r * u * w * (u + r) * (w + r) * (u + w))
    # Reference in extended precision (mpmath-free: Python fractions of the
    # series around the midpoint are overkill; use longdouble differences
    # when x, y are well separated, the derivative otherwise).
    g = lambda s: -1.0 / (np.sqrt(a + s) * r * (np.sqrt(a + s) + r))  # noqa: E731
    if abs(x - y) > 1e-3:
        ref = (g(x) - g(y)) / (x - y)
    else:
        m, h = 0.5 * (x + y), 1e-4
        ref = (g(m + h) - g(m - h)) / (2 * h)
    assert abs(gxy - ref) <= 1e-7 * abs(ref)
    # h(s) = 1/(a+s): h[x, y] = -1 / ((a+x)(a+y)).
    hxy = -1.0 / ((a + x) * (a + y))
    if abs(x - y) > 1e-3:
        assert abs(hxy - (1 / (a + x) - 1 / (a + y)) / (x - y)) <= 1e-12 * abs(hxy)


def _jacobi32(A, sweeps=8, rel=3e-8):
    A = A.astype(np.float32).copy()
    n = A.shape[0]
    U = np.eye(n, dtype=np.float32)
    thresh = np.float32(rel) * np.sqrt(np.float32((A.astype(np.float64) ** 2).sum()))
    for _ in range(sweeps):
        for pp in range(n - 1):
            for qq in range(pp + 1, n):
                apq = A[pp, qq]
                if abs(apq) <= thresh:
                    continue
                tau = (A[qq, qq] - A[pp, pp]) / (np.float32(2) * apq)
                t = np.float32(1 if tau >= 0 else -1) / (abs(tau) + np.sqrt(np.float32(1) + tau * tau))
                c = np.float32(1) / np.sqrt(np.float32(1) + t * t)
                s = t * c
                J = np.eye(n, dtype=np.float32)
                J[pp, pp] = J[qq, qq] = c
                J[pp, qq], J[qq, pp] = s, -s
                A = J.T @ A @ J
                U = U @ J
    return U.astype(np.float64)


def test_binary32_basis_refined_in_fp64_gives_fp64_matrix_functions():
    k, p = 64, 20
    dY, rho, d, a = _problem(k, p, 3)
    Yh = np.sqrt(rho)[:, None] * dY
    A = Yh @ Yh.T
    X = _jacobi32(A)
    # Cholesky QR in FP64, then the Rayleigh-Ritz matrix.
    L = np.linalg.cholesky(X.T @ X)
    Y = np.linalg.solve(L, X.T).T
    S = Y.T @ A @ Y
    s = np.diag(S)
    r = np.sqrt(a)
    u = np.sqrt(a + s)
    alpha = 1.0 / (u * (u + r))
    G = S * (u[:, None] + u[None, :] + r) * np.outer(alpha, alpha) / (r * (u[:, None] + u[None, :]))
    np.fill_diagonal(G, -alpha / r)
    H = -S / np.outer(a + s, a + s)
    np.fill_diagonal(H, 1.0 / (a + s))
    g = lambda x: ((a + x) ** -0.5 - a ** -0.5) / x  # noqa: E731
    G_ref = _fun(A, g)
    H_ref = np.linalg.inv(a * np.eye(p) + A)
    assert np.abs(Y @ G @ Y.T - G_ref).max() <= 1e-12 * np.abs(G_ref).max()
    assert np.abs(Y @ H @ Y.T - H_ref).max() <= 1e-12 * np.abs(H_ref).max()
    # The binary32 basis alone is only good to ~1e-6.
    w32 = np.diag(X.T @ A @ X)
    assert np.abs(X @ np.diag(g(w32)) @ X.T - G_ref).max() > 1e-9 * np.abs(G_ref).max()


def _refined_functions(A, X, a):
    """The analysis kernel's refinement: S' = S - E o (d_i + d_j)/2,
    first-order h(S') and g(S'), then F - E o (f_i + f_j)/2, in the basis X."""
    p = A.shape[0]
    E = X.T @ X - np.eye(p)
    S = X.T @ A @ X
    d = np.diag(S).copy()
    Sp = S - E * (d[:, None] + d[None, :]) / 2
    s = np.diag(Sp)
    r = np.sqrt(a)
    u = np.sqrt(a + s)
    alpha = 1.0 / (u * (u + r))
    G = Sp * (u[:, None] + u[None, :] + r) * np.outer(alpha, alpha) / (r * (u[:, None] + u[None, :]))
    np.fill_diagonal(G, -alpha / r)
    H = -Sp / np.outer(a + s, a + s)
    np.fill_diagonal(H, 1.0 / (a + s))
    gd, hd = np.diag(G).copy(), np.diag(H).copy()
    G = G - E * (gd[:, None] + gd[None, :]) / 2
    H = H - E * (hd[:, None] + hd[None, :]) / 2
    return G, H, np.abs(E).max()


@pytest.mark.parametrize("rel", [3e-8, 1e-6])
@pytest.mark.parametrize("k,p,seed", [(64, 20, 3), (64, 28, 4), (40, 30, 5), (64, 12, 6)])
def test_first_order_refinement_of_a_binary32_basis(k, p, seed, rel):
    """rel: the binary32 Jacobi's stopping threshold (the kernel stops at
    1e-6 of |A|_F); the remaining off-diagonal enters at second order."""
    dY, rho, d, a = _problem(k, p, seed)
    Yh = np.sqrt(rho)[:, None] * dY
    A = Yh @ Yh.T
    X = _jacobi32(A, rel=rel)
    G, H, e = _refined_functions(A, X, a)
    g = lambda x: ((a + x) ** -0.5 - a ** -0.5) / x  # noqa: E731
    G_ref = _fun(A, g)
    H_ref = np.linalg.inv(a * np.eye(p) + A)
    # Second order in the non-orthogonality (|E| ~ 5e-6 here).
    bound = max(5 * e * e, 1e-13)
    assert np.abs(X @ G @ X.T - G_ref).max() <= bound * np.abs(G_ref).max()
    assert np.abs(X @ H @ X.T - H_ref).max() <= bound * np.abs(H_ref).max()
    # Without the first-order terms the error is first order in E.
    E = X.T @ X - np.eye(p)
    S = X.T @ A @ X
    s = np.diag(S)
    assert np.abs(X @ np.diag(g(s)) @ X.T - G_ref).max() > 10 * bound * np.abs(G_ref).max()


@pytest.mark.parametrize("k,p,seed", [(160, 120, 7), (140, 128, 8)])
def test_first_order_refinement_up_to_n_128(k, p, seed):
    """The same second-order bound for the largest local problems the mixed
    path takes (n = 120, 128), where a sweep of the binary32 Jacobi is about
    twenty times as many rotations as at n = 28, at the kernels' threshold
    of 1e-6 ||A||_F."""
    test_first_order_refinement_of_a_binary32_basis(k, p, seed, 1e-6)


def _two_sum(a, b):
    f = np.float32
    s = (a + b).astype(f)
    z = (s - a).astype(f)
    return s, ((a - (s - z)).astype(f) + (b - z).astype(f)).astype(f)


def _df_acc(s, c, ah, al, y):
    """(s, c) += (ah + al) y in binary32 with an exact product error (the
    float64 product of two binary32 numbers is exact), as the kernel's FMA
    gives it."""
    f = np.float32
    p = (ah * y).astype(f)
    e = (ah.astype(np.float64) * y - p).astype(f)
    s, t = _two_sum(s, p)
    low = (al.astype(np.float64) * y + e).astype(f)  # one rounding, like an FMA
    return s, (c + (t + low).astype(f)).astype(f)


@pytest.mark.parametrize("k,p,seed", [(64, 20, 3), (40, 30, 5)])
def test_double_binary32_products_are_fp64_class(k, p, seed):
    """Y^T Y, A Y and Y^T (A Y) from binary32 arithmetic with error-free
    transformations: the basis is binary32 (exact), A is split into binary32
    halves; the results match FP64 products of the same numbers to a few
    1e-14 of |A| (plain binary32 would give ~1e-7)."""
    dY, rho, d, a = _problem(k, p, seed)
    Yh = np.sqrt(rho)[:, None] * dY
    A = Yh @ Yh.T
    X = _jacobi32(A).astype(np.float32)
    n = p
    f = np.float32
    Ah = A.astype(f)
    Al = (A - Ah.astype(np.float64)).astype(f)
    z = np.zeros((n, n), f)
    s, c = z.copy(), z.copy()
    for r in range(n):  # W = A X
        s, c = _df_acc(s, c, Ah[:, r][:, None], Al[:, r][:, None], X[r, :][None, :])
    Wh, Wl = _two_sum(s, c)
    s, c, s2, c2 = z.copy(), z.copy(), z.copy(), z.copy()
    for r in range(n):  # S = X^T W, E = X^T X - I
        s, c = _df_acc(s, c, Wh[r, :][None, :], Wl[r, :][None, :], X[r, :][:, None])
        s2, c2 = _df_acc(s2, c2, X[r, :][None, :], z[r, :][None, :], X[r, :][:, None])
    S = s.astype(np.float64) + c
    E = s2.astype(np.float64) + c2 - np.eye(n)
    Xd = X.astype(np.float64)
    scale = np.abs(A).max()
    assert np.abs(S - Xd.T @ A @ Xd).max() <= 1e-13 * scale
    assert np.abs(E - (Xd.T @ Xd - np.eye(n))).max() <= 1e-13
    # The same sums in plain binary32 are orders of magnitude worse.
    S32 = (X.T @ (Ah @ X)).astype(np.float64)
    assert np.abs(S32 - Xd.T @ A @ Xd).max() > 1e-9 * scale


@pytest.mark.parametrize("k,p,seed", [(32, 104, 11), (64, 200, 12), (128, 90, 13)])
def test_double_binary32_gram_is_fp64_class(k, p, seed):
    """The arithmetic of the double-binary32 Gram pass (LBM_PROD_DF32):
    C = sum_r rho_r y_r y_r^T with the FP64 rows and weights split into
    binary32 halves, each lane's weighted value rho y_n formed in
    double-binary32 (rh yh with its exact product error, plus rh yl and
    rl yh, renormalised into (wy)h + (wy)l), yh (wy)h accumulated with its
    exact product error, the cross terms yh (wy)l and yl (wy)h in binary32,
    yl (wy)l dropped. It must match the FP64 Gram to a few 1e-13 of |C|
    over sums of up to 200 rows (the binary32 compensation term limits it;
    binary32 products give ~1e-7)."""
    dY, rho, d, a = _problem(k, p, seed)
    f = np.float32
    Yh = dY.astype(f)
    Yl = (dY - Yh.astype(np.float64)).astype(f)
    s = np.zeros((k, k), f)
    c = np.zeros((k, k), f)
    d64 = np.float64
    for r in range(p):
        # rho y_n in double-binary32, one value per output column n; each
        # binary32 rounding is taken from the exact FP64 value (a product
        # of two binary32 numbers is exact in FP64).
        rh = f(rho[r])
        rl = f(rho[r] - d64(rh))
        yh, yl = Yh[r, :], Yl[r, :]
        pr = (rh * yh).astype(f)
        e = (d64(rh) * yh.astype(d64) - pr.astype(d64)).astype(f)  # exact error of rh yh
        e = (d64(rl) * yh.astype(d64) + e.astype(d64)).astype(f)
        e = (d64(rh) * yl.astype(d64) + e.astype(d64)).astype(f)
        wh = (pr + e).astype(f)
        wl = (e - (wh - pr).astype(f)).astype(f)
        s, c = _df_acc(s, c, Yh[r, :][:, None], Yl[r, :][:, None], wh[None, :])
        # c += yh (wy)l as one FMA.
        c = (c.astype(np.float64) + Yh[r, :][:, None].astype(np.float64) * wl[None, :]).astype(f)
    C_df = s.astype(np.float64) + c
    C_ref = (dY.T * rho) @ dY
    scale = np.abs(C_ref).max()
    assert np.abs(C_df - C_ref).max() <= 5e-13 * scale
    C32 = ((dY.T * rho).astype(f) @ dY.astype(f)).astype(np.float64)
    assert np.abs(C32 - C_ref).max() > 1e-10 * scale


def _jacobi64(A, U, rel=3e-8, max_sweeps=30):
    """Cyclic FP64 Jacobi from (A, U) with the kernels' stopping rule (no
    rotation above rel ||A||_F); returns U, A and the sweeps counted with
    the last, rotation-free one."""
    A = A.copy()
    U = U.copy()
    n = A.shape[0]
    thresh = rel * np.sqrt((A * A).sum())
    for sweep in range(max_sweeps):
        rotated = False
        for pp in range(n - 1):
            for qq in range(pp + 1, n):
                apq = A[pp, qq]
                if abs(apq) <= thresh:
                    continue
                rotated = True
                th, ph = A[qq, qq] - A[pp, pp], 2.0 * apq
                rr = np.hypot(th, ph)
                t = ph / (th + rr if th >= 0 else th - rr)
                cs = 1.0 / np.sqrt(1.0 + t * t)
                sn = t * cs
                J = np.array([[cs, sn], [-sn, cs]])
                A[:, [pp, qq]] = A[:, [pp, qq]] @ J
                A[[pp, qq], :] = J.T @ A[[pp, qq], :]
                U[:, [pp, qq]] = U[:, [pp, qq]] @ J
        if not rotated:
            return U, A, sweep + 1
    return U, A, -1


@pytest.mark.parametrize("k,p,seed", [(64, 28, 21), (64, 20, 22), (48, 28, 23)])
def test_fp64_jacobi_from_an_orthonormalised_binary32_basis(k, p, seed):
    """The FP64 run path: a binary32 Jacobi basis Y (stopped at 1e-6 of
    ||A||_F) made orthonormal on the binary32 units (E = Y^T Y - I from
    exact products summed in double-binary32, the correction Y E in
    binary32, Y1 = Y - Y E / 2 in FP64), then the FP64 Jacobi from
    A' = Y1^T A Y1 with U = Y1. Y1 is orthonormal to second order in the
    basis' binary32 non-orthogonality (~1e-13), the FP64
    Jacobi needs far fewer sweeps than from the identity, and the matrix
    functions from it are FP64-accurate."""
    dY, rho, d, a = _problem(k, p, seed)
    Yh = np.sqrt(rho)[:, None] * dY
    A = Yh @ Yh.T
    f = np.float32
    Y = _jacobi32(A, rel=1e-6).astype(f)
    n = p
    # Kernel J's own first-order re-orthonormalisation in binary32, which
    # leaves |Y^T Y - I| at the binary32 level (~1e-7).
    E32 = (Y.T @ Y - np.eye(n, dtype=f)).astype(f)
    Y = (Y - f(0.5) * (Y @ E32)).astype(f)
    e0 = np.abs(Y.astype(np.float64).T @ Y.astype(np.float64) - np.eye(n)).max()
    assert e0 < 1e-6
    z = np.zeros((n, n), f)
    s, c = z.copy(), z.copy()
    for r in range(n):
        s, c = _df_acc(s, c, Y[r, :][:, None], z[r, :][:, None], Y[r, :][None, :])
    E = (s.astype(np.float64) + c - np.eye(n)).astype(f)
    YE = (Y @ E).astype(np.float64)  # binary32 products and sums
    Y1 = Y.astype(np.float64) - 0.5 * YE
    # One step leaves the non-orthogonality at second order in e0.
    assert np.abs(Y1.T @ Y1 - np.eye(n)).max() <= n * e0 * e0 + 1e-13
    Ap = Y1.T @ A @ Y1
    Ap = 0.5 * (Ap + Ap.T)
    U, S, sweeps = _jacobi64(Ap, Y1)
    _, _, cold = _jacobi64(A, np.eye(n))
    assert 0 < sweeps <= 3 and sweeps < cold
    # Matrix functions from the FP64 eigenpairs (first order in the
    # remaining off-diagonal, as the kernel takes them).
    S = U.T @ A @ U
    sd = np.diag(S)
    r = np.sqrt(a)
    u = np.sqrt(a + sd)
    alpha = 1.0 / (u * (u + r))
    G = S * (u[:, None] + u[None, :] + r) * np.outer(alpha, alpha) / (r * (u[:, None] + u[None, :]))
    np.fill_diagonal(G, -alpha / r)
    H = -S / np.outer(a + sd, a + sd)
    np.fill_diagonal(H, 1.0 / (a + sd))
    g = lambda x: ((a + x) ** -0.5 - a ** -0.5) / x  # noqa: E731
    G_ref = _fun(A, g)
    H_ref = np.linalg.inv(a * np.eye(p) + A)
    assert np.abs(U @ G @ U.T - G_ref).max() <= 1e-12 * np.abs(G_ref).max()
    assert np.abs(U @ H @ U.T - H_ref).max() <= 1e-12 * np.abs(H_ref).max()
