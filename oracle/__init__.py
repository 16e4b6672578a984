"""CPU oracle for the LBM-LETKF cycle (arXiv 2308.03972).

TEST INFRASTRUCTURE ONLY. The oracle is a plain FP64 C library (``lbm.c``,
``eig.c``, ``letkf.c``, ``diag.c``) with this thin ctypes/numpy wrapper. It shares no code
with the CUDA library and imports nothing from the product package. Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
load it.

Functions mirror ``oracle.h``; every array argument is a C-contiguous
float64/int32 numpy array with the layouts documented there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ("lbm.c", "eig.c", "letkf.c", "diag.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblbm_letkf_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        sig = {
            "orc_d2q9": (None, [P, P, P]),
            "orc_equilibrium": (None, [D, D, D, P]),
            "orc_lbm_step": (None, [I, I, I, P, P, P, D, D, D]),
            "orc_lbm_moments": (None, [I, I, I, P, P, P, P]),
            "orc_set_equilibrium": (None, [I, I, I, P, P, P, P]),
            "orc_observe": (None, [I, I, I, P, I, P, P, P]),
            "orc_gaspari_cohn": (D, [D]),
            "orc_sym_eig": (I, [I, P, P, P]),
            "orc_letkf_transform": (I, [I, I, P, P, P, D, P, P]),
            "orc_letkf_update": (I, [I, I, P, I, P, P, P, D]),
            "orc_local_obs": (I, [I, I, I, I, I, P, P, D, D, D, P, P]),
            "orc_letkf_analyze": (I, [I, I, I, P, I, P, P, P, P, D, D, D, D, I, P]),
            "orc_num_threads": (I, []),
            "orc_set_num_threads": (None, [I]),
            "orc_nudge": (None, [I, I, I, P, I, I, P, P, P, D]),
            "orc_energy_spectrum": (None, [I, I, I, P, I, P]),
            "orc_observe_vars": (None, [I, I, I, P, I, P, P, I, P]),
            "orc_local_obs_vars": (I, [I, I, I, I, I, P, P, I, P, D, P, P]),
            "orc_letkf_analyze_vars": (I, [I, I, I, P, I, P, P, I, P, P, D, D, I, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def d2q9():
    """Return (cx, cy, w) of the D2Q9 set as the oracle defines it."""
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    _load().orc_d2q9(_p(cx), _p(cy), _p(w))
    return cx, cy, w


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9, np.float64)
    _load().orc_equilibrium(float(rho), float(ux), float(uy), _p(out))
    return out


def lbm_step(f: np.ndarray, force: np.ndarray, tau0: float, cs_smag: float, mu: float) -> np.ndarray:
    """One collide+push step. f: [9][ny][nx][k]; force: [2][ny][nx]."""
    f = _f64(f)
    force = _f64(force)
    _, ny, nx, k = f.shape
    assert force.shape == (2, ny, nx)
    out = np.empty_like(f)
    _load().orc_lbm_step(nx, ny, k, _p(f), _p(out), _p(force), float(tau0), float(cs_smag), float(mu))
    return out


def lbm_run(f: np.ndarray, force: np.ndarray, tau0: float, cs_smag: float, mu: float, nsteps: int) -> np.ndarray:
    f = _f64(f).copy()
    for _ in range(nsteps):
        f = lbm_step(f, force, tau0, cs_smag, mu)
    return f


def moments(f: np.ndarray):
    """Return rho, u, v, each [ny][nx][k]."""
    f = _f64(f)
    _, ny, nx, k = f.shape
    rho = np.empty((ny, nx, k))
    u = np.empty((ny, nx, k))
    v = np.empty((ny, nx, k))
    _load().orc_lbm_moments(nx, ny, k, _p(f), _p(rho), _p(u), _p(v))
    return rho, u, v


def set_equilibrium(rho: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """f^eq(rho, u, v) for arrays [ny][nx][k] -> f [9][ny][nx][k]."""
    rho, u, v = _f64(rho), _f64(u), _f64(v)
    ny, nx, k = rho.shape
    f = np.empty((9, ny, nx, k))
    _load().orc_set_equilibrium(nx, ny, k, _p(rho), _p(u), _p(v), _p(f))
    return f


def observe(f: np.ndarray, ix, iy) -> np.ndarray:
    """Yf [2*npts][k]: row 2j = u at point j, row 2j+1 = v."""
    f = _f64(f)
    ix, iy = _i32(ix), _i32(iy)
    _, ny, nx, k = f.shape
    Y = np.empty((2 * len(ix), k))
    _load().orc_observe(nx, ny, k, _p(f), len(ix), _p(ix), _p(iy), _p(Y))
    return Y


def gaspari_cohn(d: float) -> float:
    return _load().orc_gaspari_cohn(float(d))


def sym_eig(A: np.ndarray):
    A = _f64(A)
    n = A.shape[0]
    lam = np.empty(n)
    Q = np.empty((n, n))
    st = _load().orc_sym_eig(n, _p(A), _p(lam), _p(Q))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return lam, Q


def letkf_transform(dY: np.ndarray, rloc: np.ndarray, d: np.ndarray, beta: float):
    """Return (wbar[k], W[k][k]) for local dY [p][k], rloc [p], d [p]."""
    dY, rloc, d = _f64(dY), _f64(rloc), _f64(d)
    p, k = dY.shape
    wbar = np.empty(k)
    W = np.empty((k, k))
    st = _load().orc_letkf_transform(k, p, _p(dY), _p(rloc), _p(d), float(beta), _p(wbar), _p(W))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return wbar, W


def letkf_update(X: np.ndarray, dY: np.ndarray, rloc: np.ndarray, d: np.ndarray, beta: float) -> np.ndarray:
    """Analysis of X [nrows][k] with local dY [p][k]; returns a new array."""
    X = _f64(X).copy()
    dY, rloc, d = _f64(dY), _f64(rloc), _f64(d)
    nrows, k = X.shape
    p = dY.shape[0] if dY.size else 0
    st = _load().orc_letkf_update(nrows, k, _p(X), p, _p(dY.reshape(p, k) if p else np.zeros((1, k))),
                                  _p(rloc if p else np.zeros(1)), _p(d if p else np.zeros(1)), float(beta))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return X


def local_obs(nx, ny, x, y, ix, iy, sigma_u, sigma_v, d_cut):
    ix, iy = _i32(ix), _i32(iy)
    idx = np.zeros(2 * len(ix), np.int32)
    rl = np.zeros(2 * len(ix), np.float64)
    p = _load().orc_local_obs(nx, ny, x, y, len(ix), _p(ix), _p(iy), float(sigma_u), float(sigma_v),
                              float(d_cut), _p(idx), _p(rl))
    return idx[:p].copy(), rl[:p].copy()


def letkf_analyze(f: np.ndarray, ix, iy, yo_u, yo_v, sigma_u, sigma_v, d_cut, beta, points=None) -> np.ndarray:
    """LETKF analysis of f [9][ny][nx][k]; returns a new array.

    points: optional int array of cell indices y*nx+x; only those cells are
    updated (the rest are copied unchanged)."""
    f = _f64(f).copy()
    ix, iy = _i32(ix), _i32(iy)
    yo_u, yo_v = _f64(yo_u), _f64(yo_v)
    _, ny, nx, k = f.shape
    if points is None:
        npoints, pts = -1, np.zeros(1, np.int32)
    else:
        pts = _i32(points)
        npoints = len(pts)
    st = _load().orc_letkf_analyze(nx, ny, k, _p(f), len(ix), _p(ix), _p(iy), _p(yo_u), _p(yo_v),
                                   float(sigma_u), float(sigma_v), float(d_cut), float(beta), npoints, _p(pts))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return f


def observe_vars(f: np.ndarray, ix, iy, nvar: int) -> np.ndarray:
    """Yf [nvar*npts][k]: rows u, v (and rho when nvar = 3) of each point."""
    f = _f64(f)
    ix, iy = _i32(ix), _i32(iy)
    _, ny, nx, k = f.shape
    Y = np.empty((nvar * len(ix), k))
    _load().orc_observe_vars(nx, ny, k, _p(f), len(ix), _p(ix), _p(iy), int(nvar), _p(Y))
    return Y


def local_obs_vars(nx, ny, x, y, ix, iy, sigma, d_cut):
    """Local set with len(sigma) variables per point."""
    ix, iy = _i32(ix), _i32(iy)
    sigma = _f64(sigma)
    nvar = len(sigma)
    idx = np.zeros(nvar * len(ix), np.int32)
    rl = np.zeros(nvar * len(ix), np.float64)
    p = _load().orc_local_obs_vars(nx, ny, x, y, len(ix), _p(ix), _p(iy), nvar, _p(sigma),
                                   float(d_cut), _p(idx), _p(rl))
    return idx[:p].copy(), rl[:p].copy()


def letkf_analyze_vars(f: np.ndarray, ix, iy, yo, sigma, d_cut, beta, points=None) -> np.ndarray:
    """LETKF analysis with len(sigma) observed variables per point (u, v[,
    rho]); yo [npts][nvar]. Returns a new array."""
    f = _f64(f).copy()
    ix, iy = _i32(ix), _i32(iy)
    sigma = _f64(sigma)
    nvar = len(sigma)
    yo = _f64(yo).reshape(len(ix), nvar)
    _, ny, nx, k = f.shape
    if points is None:
        npoints, pts = -1, np.zeros(1, np.int32)
    else:
        pts = _i32(points)
        npoints = len(pts)
    st = _load().orc_letkf_analyze_vars(nx, ny, k, _p(f), len(ix), _p(ix), _p(iy), nvar, _p(yo),
                                        _p(sigma), float(d_cut), float(beta), npoints, _p(pts))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return f


def nudge(f: np.ndarray, rho_o, u_o, v_o, gamma: float) -> np.ndarray:
    """Nudging of f [9][ny][nx][k] toward f^eq of the observed fields
    [noy][nox] on the uniform lattice (bilinear interpolation); new array."""
    f = _f64(f).copy()
    rho_o, u_o, v_o = _f64(rho_o), _f64(u_o), _f64(v_o)
    _, ny, nx, k = f.shape
    noy, nox = rho_o.shape
    assert nx % nox == 0 and ny % noy == 0
    _load().orc_nudge(nx, ny, k, _p(f), nox, noy, _p(rho_o), _p(u_o), _p(v_o), float(gamma))
    return f


def spectrum_shells(nx: int, ny: int) -> int:
    """Number of shells that hold every wavenumber of an nx x ny lattice."""
    return int(np.floor(np.hypot(nx // 2, ny // 2) + 0.5)) + 1


def energy_spectrum(f: np.ndarray, nshells: int | None = None) -> np.ndarray:
    """Member-averaged energy spectrum E[s] of f [9][ny][nx][k] (shells
    s = floor(|k'| + 1/2))."""
    f = _f64(f)
    _, ny, nx, k = f.shape
    if nshells is None:
        nshells = spectrum_shells(nx, ny)
    E = np.zeros(nshells)
    _load().orc_energy_spectrum(nx, ny, k, _p(f), int(nshells), _p(E))
    return E


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads the oracle's OpenMP loops use from now on (n >= 1)."""
    _load().orc_set_num_threads(int(n))
