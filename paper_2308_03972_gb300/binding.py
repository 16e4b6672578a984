"""ctypes binding of the C ABI in ``include/lbm_letkf.h``.

Argument marshalling only: every step of the cycle runs in the CUDA library.
Functions keep the C names. Array arguments may be numpy arrays (host memory,
float64/int32, C-contiguous) or torch CUDA tensors (device memory, float64,
contiguous); the pointer kind is inferred. A nonzero status raises
``LbmError`` carrying the status code and the library's message.

The library must have been built (``python -m paper_2308_03972_gb300.build``
or ``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ENOCONV = range(6)
LBM_FP64, LBM_MIXED = 0, 1
LBM_PTR_HOST, LBM_PTR_DEVICE = 0, 1
LBM_PROD_FP64, LBM_PROD_FP32, LBM_PROD_TF32, LBM_PROD_BF16, LBM_PROD_DF32 = range(5)

STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_EDIVERGED", 5: "LBM_ENOCONV"}

# Every entry point the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", _I), ("ny", _I), ("members", _I), ("tau0", _D), ("cs_smag", _D),
                ("mu", _D), ("precision", _I), ("stream", _P)]


class lbm_window(ctypes.Structure):
    _fields_ = [("nsteps", _I), ("obs_every", _I), ("checkpoint_every", _I), ("npts", _I),
                ("ix", _P), ("iy", _P), ("yo_u", _P), ("yo_v", _P), ("sigma_u", _D), ("sigma_v", _D)]


SIGNATURES = {
    "lbm_init": (_I, [ctypes.POINTER(lbm_config), _P, _P, _I, ctypes.POINTER(_P)]),
    "lbm_set_equilibrium": (_I, [_P, _P, _P, _P, _I]),
    "lbm_forecast": (_I, [_P, _I]),
    "lbm_moments": (_I, [_P, _P, _P, _P, _I]),
    "lbm_mean_velocity": (_I, [_P, _P, _P, _I]),
    "lbm_velocity_rmse": (_I, [_P, _P, _P, _I]),
    "lbm_energy_spectrum": (_I, [_P, _P, _I, _I]),
    "letkf_observe": (_I, [_P, _I, _P, _P, _P, _P, _D, _D]),
    "letkf_observe_rho": (_I, [_P, _I, _P, _P, _P, _P, _P, _D, _D, _D]),
    "letkf_analyze": (_I, [_P, _D, _D]),
    "letkf_probe_transform": (_I, [_P, _D, _D, _I, _P, _P, _I]),
    "lbm_set_closure": (_I, [_P, _D]),
    "letkf_set_products": (_I, [_P, _I]),
    "letkf_set_run_length": (_I, [_P, _I]),
    "letkf_set_run_pipeline": (_I, [_P, _I]),
    "letkf_sweep_stats": (_I, [_P, _I, _P]),
    "lbm_misfit": (_I, [_P, ctypes.POINTER(lbm_window), _P]),
    "lbm_misfit_gradient": (_I, [_P, ctypes.POINTER(lbm_window), _P, _P, _P, _P, _P, _I]),
    "lbm_nudge": (_I, [_P, _I, _I, _P, _P, _P, _D]),
    "lbm_get_f": (_I, [_P, _P, _I]),
    "lbm_set_f": (_I, [_P, _P, _I]),
    "lbm_sync": (_I, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_destroy": (None, [_P]),
    "lbm_batch_create": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "lbm_batch_forecast": (_I, [_P, _I]),
    "lbm_batch_autotune": (_I, [_P, _P, _P]),
    "lbm_batch_autotune_analysis": (_I, [_P, _P, _P, _P, _P]),
    "lbm_batch_cycle": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _I]),
    "lbm_batch_sync": (_I, [_P]),
    "lbm_batch_set_barrier": (_I, [_P, ctypes.c_longlong, _I]),
    "lbm_batch_set_analysis_form": (_I, [_P, _P]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_batch_destroy": (None, [_P]),
    "letkf_analyze_noalloc": (_I, [_P, _I, _I, _I, _I, _P, _P, _P, _P, _D, _D, _D, _D, _P]),
}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: build it with "
                           "`python -m paper_2308_03972_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arr(a, dtype=np.float64, writable=False):
    """Return (pointer, ptr_kind, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, LBM_PTR_HOST, None
    if _is_torch(a):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % want)
        kind = LBM_PTR_DEVICE if a.is_cuda else LBM_PTR_HOST
        return ctypes.c_void_p(a.data_ptr()), kind, a
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        if writable:
            raise TypeError("output must be a C-contiguous %s numpy array or tensor" % np.dtype(dtype))
        a = np.ascontiguousarray(a, dtype=dtype)
    if writable and not a.flags.writeable:
        raise TypeError("output array is read-only")
    return a.ctypes.data_as(ctypes.c_void_p), LBM_PTR_HOST, a


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return ks.pop() if ks else LBM_PTR_HOST


def _check(ctx, status):
    if status != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(status, msg.decode() if msg else "")


def default_stream():
    """The current torch CUDA stream handle, or None (legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def lbm_init(nx, ny, members, tau0, cs_smag, mu, precision=LBM_FP64, f0=None, force=None,
             stream="current"):
    """Create a context; returns its handle (a ctypes void pointer)."""
    lib = load()
    if stream == "current":
        stream = default_stream()
    cfg = lbm_config(int(nx), int(ny), int(members), float(tau0), float(cs_smag), float(mu),
                     int(precision), ctypes.c_void_p(stream) if stream else None)
    pf, kf, _a = _arr(f0)
    pg, kg, _b = _arr(force)
    kind = _kind(kf if f0 is not None else None, kg if force is not None else None)
    out = ctypes.c_void_p()
    st = lib.lbm_init(ctypes.byref(cfg), pf, pg, kind, ctypes.byref(out))
    _check(None, st)
    return out


def lbm_set_equilibrium(ctx, rho, u, v):
    pr, kr, _a = _arr(rho)
    pu, ku, _b = _arr(u)
    pv, kv, _c = _arr(v)
    kind = _kind(kr if rho is not None else None, ku, kv)
    _check(ctx, load().lbm_set_equilibrium(ctx, pr, pu, pv, kind))


def lbm_forecast(ctx, nsteps):
    _check(ctx, load().lbm_forecast(ctx, int(nsteps)))


def lbm_moments(ctx, rho=None, u=None, v=None):
    """Fill the given output arrays [ny][nx][members] (numpy or CUDA tensors)."""
    pr, kr, _a = _arr(rho, writable=True)
    pu, ku, _b = _arr(u, writable=True)
    pv, kv, _c = _arr(v, writable=True)
    kind = _kind(*(k for a, k in ((rho, kr), (u, ku), (v, kv)) if a is not None))
    _check(ctx, load().lbm_moments(ctx, pr, pu, pv, kind))


def lbm_mean_velocity(ctx, u=None, v=None):
    """Fill the given ensemble-mean outputs [ny][nx] (numpy or CUDA tensors)."""
    pu, ku, _b = _arr(u, writable=True)
    pv, kv, _c = _arr(v, writable=True)
    kind = _kind(*(k for a, k in ((u, ku), (v, kv)) if a is not None))
    _check(ctx, load().lbm_mean_velocity(ctx, pu, pv, kind))


def spectrum_shells(nx: int, ny: int) -> int:
    """Shell count that holds every wavenumber of an nx x ny lattice."""
    return int(np.floor(np.hypot(nx // 2, ny // 2) + 0.5)) + 1


def lbm_energy_spectrum(ctx, E):
    """Fill E [nshells] (numpy or CUDA tensor) with the member-averaged
    shell energy spectrum."""
    pe, ke, _b = _arr(E, writable=True)
    _check(ctx, load().lbm_energy_spectrum(ctx, pe, int(E.numel() if _is_torch(E) else E.size), ke))


def letkf_observe(ctx, ix, iy, yo_u, yo_v, sigma_u, sigma_v):
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    yo_u = np.ascontiguousarray(yo_u, dtype=np.float64)
    yo_v = np.ascontiguousarray(yo_v, dtype=np.float64)
    n = len(ix)
    if not (len(iy) == len(yo_u) == len(yo_v) == n):
        raise ValueError("observation arrays differ in length")
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(ctx, load().letkf_observe(ctx, n, p(ix), p(iy), p(yo_u), p(yo_v), float(sigma_u),
                                     float(sigma_v)))


def letkf_observe_rho(ctx, ix, iy, yo_u, yo_v, yo_rho, sigma_u, sigma_v, sigma_rho):
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    yo_u = np.ascontiguousarray(yo_u, dtype=np.float64)
    yo_v = np.ascontiguousarray(yo_v, dtype=np.float64)
    yo_rho = np.ascontiguousarray(yo_rho, dtype=np.float64)
    n = len(ix)
    if not (len(iy) == len(yo_u) == len(yo_v) == len(yo_rho) == n):
        raise ValueError("observation arrays differ in length")
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(ctx, load().letkf_observe_rho(ctx, n, p(ix), p(iy), p(yo_u), p(yo_v), p(yo_rho),
                                         float(sigma_u), float(sigma_v), float(sigma_rho)))


def letkf_sweep_stats(ctx, enable, read=False):
    """Enable/disable sweep counting; with read=True return the 32-bin
    histogram (and reset it)."""
    h = np.zeros(32, np.int32) if read else None
    _check(ctx, load().letkf_sweep_stats(ctx, 1 if enable else 0,
                                         h.ctypes.data_as(ctypes.c_void_p) if read else None))
    return h


def letkf_set_products(ctx, mode):
    _check(ctx, load().letkf_set_products(ctx, int(mode)))


def letkf_set_run_length(ctx, run_len):
    _check(ctx, load().letkf_set_run_length(ctx, int(run_len)))


def letkf_set_run_pipeline(ctx, runs):
    _check(ctx, load().letkf_set_run_pipeline(ctx, int(runs)))


def lbm_set_closure(ctx, cs_smag):
    _check(ctx, load().lbm_set_closure(ctx, float(cs_smag)))


class Window:
    """Observation window of the misfit (the C struct lbm_window with its
    arrays kept alive): yo_u, yo_v [nsteps // obs_every][npts]."""

    def __init__(self, nsteps, obs_every, ix, iy, yo_u, yo_v, sigma_u, sigma_v, checkpoint_every=20):
        self.ix = np.ascontiguousarray(ix, dtype=np.int32)
        self.iy = np.ascontiguousarray(iy, dtype=np.int32)
        nt = int(nsteps) // int(obs_every)
        self.yo_u = np.ascontiguousarray(yo_u, dtype=np.float64).reshape(nt, len(self.ix))
        self.yo_v = np.ascontiguousarray(yo_v, dtype=np.float64).reshape(nt, len(self.ix))
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self.c = lbm_window(int(nsteps), int(obs_every), int(checkpoint_every), len(self.ix), p(self.ix),
                            p(self.iy), p(self.yo_u), p(self.yo_v), float(sigma_u), float(sigma_v))


def lbm_misfit(ctx, win: Window, members: int):
    J = np.zeros(members)
    _check(ctx, load().lbm_misfit(ctx, ctypes.byref(win.c), J.ctypes.data_as(ctypes.c_void_p)))
    return J


def lbm_misfit_gradient(ctx, win: Window, members: int, weights=None, grad_f0=None, dcs=None):
    """Return (J [k], grad_cs [k]); grad_f0 (float64 [9][ny][nx][k]) and dcs
    (float64 [1], dF/dC_s) are filled in place when given. weights, grad_f0
    and dcs are numpy arrays or CUDA tensors (all of one kind)."""
    J = np.zeros(members)
    gcs = np.zeros(members)
    pw, kw, _kw = _arr(weights)
    pg, kg, _keep = _arr(grad_f0, writable=True)
    pd, kd, _kd = _arr(dcs, writable=True)
    kind = _kind(kw if weights is not None else None, kg if grad_f0 is not None else None,
                 kd if dcs is not None else None)
    _check(ctx, load().lbm_misfit_gradient(ctx, ctypes.byref(win.c), pw, J.ctypes.data_as(ctypes.c_void_p),
                                           pg, gcs.ctypes.data_as(ctypes.c_void_p), pd, kind))
    return J, gcs


def lbm_velocity_rmse(ctx, truth_ctx):
    """Ensemble-mean velocity RMSE of ctx against truth_ctx (a float)."""
    r = np.zeros(1)
    _check(ctx, load().lbm_velocity_rmse(ctx, truth_ctx, r.ctypes.data_as(ctypes.c_void_p), LBM_PTR_HOST))
    return float(r[0])


def letkf_analyze(ctx, d_cut, beta):
    _check(ctx, load().letkf_analyze(ctx, float(d_cut), float(beta)))


def letkf_probe_transform(ctx, d_cut, beta, cells, members):
    """T [len(cells)][members][members] (numpy, FP64): the mixed analysis'
    transform at the grid points `cells` (y * nx + x), state unchanged."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    T = np.zeros((len(cells), members, members))
    _check(ctx, load().letkf_probe_transform(ctx, float(d_cut), float(beta), len(cells),
                                             cells.ctypes.data_as(ctypes.c_void_p),
                                             T.ctypes.data_as(ctypes.c_void_p), LBM_PTR_HOST))
    return T


def lbm_nudge(ctx, rho_o, u_o, v_o, gamma):
    """Nudge every member toward f^eq of observed fields [nobs_y][nobs_x]."""
    rho_o = np.ascontiguousarray(rho_o, dtype=np.float64)
    u_o = np.ascontiguousarray(u_o, dtype=np.float64)
    v_o = np.ascontiguousarray(v_o, dtype=np.float64)
    if not (rho_o.shape == u_o.shape == v_o.shape) or rho_o.ndim != 2:
        raise ValueError("observation fields must share one 2-d shape [nobs_y][nobs_x]")
    noy, nox = rho_o.shape
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(ctx, load().lbm_nudge(ctx, nox, noy, p(rho_o), p(u_o), p(v_o), float(gamma)))


def lbm_get_f(ctx, out):
    po, ko, _a = _arr(out, writable=True)
    _check(ctx, load().lbm_get_f(ctx, po, ko))
    return out


def lbm_set_f(ctx, f):
    pf, kf, _a = _arr(f)
    _check(ctx, load().lbm_set_f(ctx, pf, kf))


def lbm_sync(ctx):
    _check(ctx, load().lbm_sync(ctx))


def lbm_last_error(ctx) -> str:
    msg = load().lbm_last_error(ctx)
    return msg.decode() if msg else ""


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


def letkf_analyze_noalloc(f, ix, iy, yo_u, yo_v, sigma_u, sigma_v, d_cut, beta, stream="current"):
    """Allocation-free analysis of a caller-owned FP64 CUDA tensor
    f [9][ny][nx][members] in place; observations are host arrays."""
    if not _is_torch(f) or not f.is_cuda or f.dim() != 4:
        raise TypeError("f must be a 4-d CUDA float64 tensor [9][ny][nx][members]")
    import torch

    if f.device.index != torch.cuda.current_device():
        raise ValueError("f must be on the current CUDA device (the scratch address and the stream are "
                         "the current device's)")
    pf, _, _a = _arr(f)
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    yo_u = np.ascontiguousarray(yo_u, dtype=np.float64)
    yo_v = np.ascontiguousarray(yo_v, dtype=np.float64)
    if not (len(ix) == len(iy) == len(yo_u) == len(yo_v)):
        raise ValueError("ix, iy, yo_u and yo_v must have the same length")
    if stream == "current":
        stream = default_stream()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _, ny, nx, k = f.shape
    st = load().letkf_analyze_noalloc(pf, nx, ny, k, len(ix), p(ix), p(iy), p(yo_u), p(yo_v),
                                      float(sigma_u), float(sigma_v), float(d_cut), float(beta),
                                      ctypes.c_void_p(stream) if stream else None)
    _check(None, st)


class Ensemble:
    """Owns one context: the C ABI calls as methods, destroyed on close()."""

    def __init__(self, nx, ny, members, tau0=0.55, cs_smag=0.2, mu=0.0, precision=LBM_FP64,
                 f0=None, force=None, stream="current"):
        self.nx, self.ny, self.members = int(nx), int(ny), int(members)
        self.precision = precision
        self.ctx = lbm_init(nx, ny, members, tau0, cs_smag, mu, precision, f0, force, stream)

    def set_equilibrium(self, rho, u, v):
        lbm_set_equilibrium(self.ctx, rho, u, v)

    def forecast(self, nsteps):
        lbm_forecast(self.ctx, nsteps)

    def moments(self, rho=None, u=None, v=None):
        lbm_moments(self.ctx, rho, u, v)

    def moments_host(self):
        shape = (self.ny, self.nx, self.members)
        rho, u, v = np.empty(shape), np.empty(shape), np.empty(shape)
        lbm_moments(self.ctx, rho, u, v)
        return rho, u, v

    def mean_velocity(self, u=None, v=None):
        if u is None and v is None:
            u = np.empty((self.ny, self.nx))
            v = np.empty((self.ny, self.nx))
        lbm_mean_velocity(self.ctx, u, v)
        return u, v

    def energy_spectrum(self, E=None):
        if E is None:
            E = np.zeros(spectrum_shells(self.nx, self.ny))
        lbm_energy_spectrum(self.ctx, E)
        return E

    def observe(self, ix, iy, yo_u, yo_v, sigma_u, sigma_v):
        letkf_observe(self.ctx, ix, iy, yo_u, yo_v, sigma_u, sigma_v)

    def sweep_stats(self, enable, read=False):
        return letkf_sweep_stats(self.ctx, enable, read)

    def set_products(self, mode):
        letkf_set_products(self.ctx, mode)

    def set_run_length(self, run_len):
        letkf_set_run_length(self.ctx, run_len)

    def set_run_pipeline(self, runs):
        letkf_set_run_pipeline(self.ctx, runs)

    def set_closure(self, cs_smag):
        lbm_set_closure(self.ctx, cs_smag)

    def misfit(self, win):
        return lbm_misfit(self.ctx, win, self.members)

    def misfit_gradient(self, win, weights=None, grad_f0=None):
        """(J, grad_f0, grad_cs); grad_f0 is a new numpy array unless given."""
        if grad_f0 is None:
            grad_f0 = np.zeros((9, self.ny, self.nx, self.members))
        J, gcs = lbm_misfit_gradient(self.ctx, win, self.members, weights, grad_f0)
        return J, grad_f0, gcs

    def velocity_rmse(self, truth):
        """Ensemble-mean velocity RMSE against another Ensemble (the truth)."""
        return lbm_velocity_rmse(self.ctx, truth.ctx)

    def observe_rho(self, ix, iy, yo_u, yo_v, yo_rho, sigma_u, sigma_v, sigma_rho):
        letkf_observe_rho(self.ctx, ix, iy, yo_u, yo_v, yo_rho, sigma_u, sigma_v, sigma_rho)

    def probe_transform(self, d_cut, beta, cells):
        return letkf_probe_transform(self.ctx, d_cut, beta, cells, self.members)

    def analyze(self, d_cut, beta):
        letkf_analyze(self.ctx, d_cut, beta)

    def nudge(self, rho_o, u_o, v_o, gamma):
        lbm_nudge(self.ctx, rho_o, u_o, v_o, gamma)

    def get_f(self, out=None):
        if out is None:
            out = np.empty((9, self.ny, self.nx, self.members))
        return lbm_get_f(self.ctx, out)

    def set_f(self, f):
        lbm_set_f(self.ctx, f)

    def sync(self):
        lbm_sync(self.ctx)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(b, status):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(b)
        raise LbmError(status, msg.decode() if msg else "")


class Batch:
    """Independent experiments (Ensemble objects sharing one stream and
    precision) advanced together: one persistent launch per forecast, and a
    captured CUDA graph per DA cycle."""

    def __init__(self, ensembles):
        self.ens = list(ensembles)
        self.run_batched = [1] * len(self.ens)
        arr = (_P * len(self.ens))(*[e.ctx for e in self.ens])
        out = _P()
        _bcheck(None, load().lbm_batch_create(arr, len(self.ens), ctypes.byref(out)))
        self.b = out

    def forecast(self, nsteps):
        _bcheck(self.b, load().lbm_batch_forecast(self.b, int(nsteps)))

    def autotune(self):
        t, n = ctypes.c_int(0), ctypes.c_int(0)
        _bcheck(self.b, load().lbm_batch_autotune(self.b, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def autotune_analysis(self, d_cut, beta):
        """Run length per size class of the batch's analyses, and for the
        run-path classes batched or one-by-one launches; every experiment
        must be observed. Returns each experiment's run length; the launch
        form per experiment (1 batched, 0 on its own) is left in
        `self.run_batched`."""
        n = len(self.ens)
        dc = np.ascontiguousarray(d_cut, dtype=np.float64)
        bt = np.ascontiguousarray(beta, dtype=np.float64)
        if dc.shape != (n,) or bt.shape != (n,):
            raise ValueError("d_cut and beta need one value per experiment")
        out = np.zeros(n, dtype=np.int32)
        form = np.zeros(n, dtype=np.int32)
        p = lambda a: a.ctypes.data_as(_P)  # noqa: E731
        _bcheck(self.b, load().lbm_batch_autotune_analysis(self.b, p(dc), p(bt), p(out), p(form)))
        self.run_batched = form.tolist()
        return out.tolist()

    def cycle(self, nsteps, obs, d_cut, beta, use_graph=True):
        """obs: per experiment (ix, iy, yo_u, yo_v, sigma_u, sigma_v)."""
        n = len(self.ens)
        keep = []

        def arrs(i, dt):
            a = [np.ascontiguousarray(o[i], dtype=dt) for o in obs]
            keep.extend(a)
            return (_P * n)(*[x.ctypes.data_as(_P) for x in a])
        npts = np.array([len(o[0]) for o in obs], dtype=np.int32)
        sig = np.array([[o[4], o[5]] for o in obs], dtype=np.float64).ravel()
        dc = np.ascontiguousarray(d_cut, dtype=np.float64)
        bt = np.ascontiguousarray(beta, dtype=np.float64)
        p = lambda a: a.ctypes.data_as(_P)  # noqa: E731
        _bcheck(self.b, load().lbm_batch_cycle(self.b, int(nsteps), p(npts), arrs(0, np.int32), arrs(1, np.int32),
                                               arrs(2, np.float64), arrs(3, np.float64), p(sig), p(dc), p(bt),
                                               1 if use_graph else 0))

    def set_analysis_form(self, batched):
        """Launch form of each experiment's run analysis: 1 batched, 0 on its own."""
        form = np.ascontiguousarray(batched, dtype=np.int32)
        if form.shape != (len(self.ens),):
            raise ValueError("one launch form per experiment")
        _bcheck(self.b, load().lbm_batch_set_analysis_form(self.b, form.ctypes.data_as(_P)))
        self.run_batched = form.tolist()

    def set_barrier(self, spin_limit, absent=0):
        _bcheck(self.b, load().lbm_batch_set_barrier(self.b, int(spin_limit), int(absent)))

    def sync(self):
        _bcheck(self.b, load().lbm_batch_sync(self.b))

    def close(self):
        if self.b:
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
