"""The analysis over runs of neighbouring grid points, mixed precision and FP64
(warm-started binary32 Jacobi over the union of a run's local sets, Section
3.2) against the FP64 oracle and against the chunked path (cold starts),
through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import U_RMS, norm_rel, osse_observations, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS


def _case(nx, ny, k, nox, noy, seed, steps=4):
    f = turbulent_state(oracle, nx, ny, k, seed=seed)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f = oracle.lbm_run(f, force, TAU0, CS, MU, steps)
    tu, tv = inputs.random_velocity(nx, ny, seed + 1000, U_RMS)
    ix, iy, yu, yv = osse_observations(nx, ny, nox, noy, 4, 1, tu, tv, SIGMA)
    return f, ix, iy, yu, yv


def _binary32_exact(f):
    """f whose f - w_alpha is exact in binary32 (the mixed state's storage)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4).reshape(9, 1, 1, 1)
    return (f - w).astype(np.float32).astype(np.float64) + w


def _mixed(b, f, ix, iy, yu, yv, d_cut, beta, run_len, hist=False):
    _, ny, nx, k = f.shape
    with b.Ensemble(nx, ny, k, TAU0, CS, MU, b.LBM_MIXED, f0=f) as e:
        e.set_run_length(run_len)
        if hist:
            e.sweep_stats(True)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, beta)
        out = e.get_f()
        h = e.sweep_stats(False, read=True) if hist else None
        e.sync()
    return out, h


# (nx, ny, k, obs lattice, d_cut): every grid point in observation space
# (p < k), unions of at most 32 scalars.
CASES = [
    (40, 24, 40, 4, 4, 5.0),    # unions of 8..24 scalars
    (36, 20, 64, 3, 2, 9.0),    # ragged runs at the row end (36 = 4 x 8 + 4)
    (48, 32, 33, 6, 4, 3.5),    # odd members (scalar staging of the ensemble)
    (32, 32, 64, 4, 4, 8.0),    # unions near 32
]


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", CASES)
@pytest.mark.parametrize("run_len", [1, 3, 8, 1000])
def test_runs_match_oracle(gpu, nx, ny, k, nox, noy, d_cut, run_len):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + k)
    f = _binary32_exact(f)
    got, _ = _mixed(gpu, f, ix, iy, yu, yv, d_cut, 1.05, run_len)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    # Binary32 storage and transform: the bound of the mixed analysis.
    assert norm_rel(got, ref) <= 5e-8
    assert norm_rel(ref, f) > 1e-6


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", CASES)
def test_runs_match_chunked_path(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + 2 * k)
    f = _binary32_exact(f)
    runs, _ = _mixed(gpu, f, ix, iy, yu, yv, d_cut, 1.05, 8)
    chunked, _ = _mixed(gpu, f, ix, iy, yu, yv, d_cut, 1.05, 0)
    assert norm_rel(runs, chunked) <= 5e-8


def test_warm_starts_take_fewer_sweeps(gpu):
    """Paper-scale geometry (256^2, 64 members, 8 x 8 points, d_cut = 32):
    runs of 8 grid points against one point per run (all cold)."""
    nx = ny = 256
    k = 64
    f, ix, iy, yu, yv = _case(nx, ny, k, 8, 8, seed=5, steps=1)
    _, h8 = _mixed(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 8, hist=True)
    _, h1 = _mixed(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 1, hist=True)
    assert h8.sum() == h1.sum() == nx * ny
    assert h8[31] == 0 and h1[31] == 0
    mean8 = (h8 * np.arange(32)).sum() / h8.sum()
    mean1 = (h1 * np.arange(32)).sum() / h1.sum()
    assert mean8 < 0.8 * mean1


def test_paper_scale_runs_sampled_points(gpu):
    """256^2 x 64, 8 x 8 observation points, d_cut = 32, runs of 8: sampled
    grid points against the oracle, including run starts and ends."""
    nx = ny = 256
    k = 64
    f, ix, iy, yu, yv = _case(nx, ny, k, 8, 8, seed=23, steps=1)
    f = _binary32_exact(f)
    got, _ = _mixed(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 8)
    rng = np.random.default_rng(1)
    pts = np.unique(np.concatenate([rng.integers(0, nx * ny, 120),
                                    [0, 7, 8, 255, 256 * 100 + 63, 256 * 100 + 64, nx * ny - 1]]))
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 32.0, 1.05, points=pts.astype(np.int32))
    g = got.reshape(9, nx * ny, k)[:, pts]
    r = ref.reshape(9, nx * ny, k)[:, pts]
    assert norm_rel(g, r) <= 5e-8


def test_run_length_argument(gpu):
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_MIXED) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.set_run_length(-1)
        assert err.value.code == gpu.LBM_EINVAL
        e.set_run_length(0)
        e.set_run_length(16)


# ---- double precision: the FP64 Jacobi warm-started from the run's basis --

def _fp64(b, f, ix, iy, yu, yv, d_cut, beta, run_len, hist=False):
    _, ny, nx, k = f.shape
    with b.Ensemble(nx, ny, k, TAU0, CS, MU, b.LBM_FP64, f0=f) as e:
        e.set_run_length(run_len)
        if hist:
            e.sweep_stats(True)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, beta)
        out = e.get_f()
        h = e.sweep_stats(False, read=True) if hist else None
        e.sync()
    return out, h


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", CASES)
@pytest.mark.parametrize("run_len", [1, 3, 8, 1000])
def test_fp64_runs_match_oracle(gpu, nx, ny, k, nox, noy, d_cut, run_len):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + 3 * k)
    got, _ = _fp64(gpu, f, ix, iy, yu, yv, d_cut, 1.05, run_len)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    assert norm_rel(got, ref) <= 1e-12
    assert norm_rel(ref, f) > 1e-6


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", CASES)
def test_fp64_runs_match_cold_path(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + 4 * k)
    runs, _ = _fp64(gpu, f, ix, iy, yu, yv, d_cut, 1.05, 8)
    cold, _ = _fp64(gpu, f, ix, iy, yu, yv, d_cut, 1.05, 0)
    assert norm_rel(runs, cold) <= 1e-13


def test_fp64_warm_starts_take_fewer_sweeps(gpu):
    """Paper-scale geometry: the FP64 Jacobi from the binary32 basis against
    the cold FP64 Jacobi (sweeps counted up to and including the one that
    finds convergence)."""
    nx = ny = 256
    k = 64
    f, ix, iy, yu, yv = _case(nx, ny, k, 8, 8, seed=6, steps=1)
    _, hw = _fp64(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 8, hist=True)
    _, hc = _fp64(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 0, hist=True)
    assert hw.sum() == hc.sum() == nx * ny
    assert hw[31] == 0 and hc[31] == 0
    meanw = (hw * np.arange(32)).sum() / hw.sum()
    meanc = (hc * np.arange(32)).sum() / hc.sum()
    assert meanw <= 3.0 and meanw < 0.5 * meanc


def test_fp64_paper_scale_runs_sampled_points(gpu):
    """256^2 x 64, 8 x 8 observation points, d_cut = 32, runs of 8, FP64:
    sampled grid points against the oracle at the FP64 bound."""
    nx = ny = 256
    k = 64
    f, ix, iy, yu, yv = _case(nx, ny, k, 8, 8, seed=29, steps=1)
    got, _ = _fp64(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 8)
    rng = np.random.default_rng(2)
    pts = np.unique(np.concatenate([rng.integers(0, nx * ny, 120),
                                    [0, 7, 8, 255, 256 * 100 + 63, 256 * 100 + 64, nx * ny - 1]]))
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 32.0, 1.05, points=pts.astype(np.int32))
    g = got.reshape(9, nx * ny, k)[:, pts]
    r = ref.reshape(9, nx * ny, k)[:, pts]
    assert norm_rel(g, r) <= 1e-12


# ---- ensemble-space points: kernel (A) warm-started along runs -------------

ENS_CASES = [
    (40, 32, 16, 10, 8, 8.0),   # every point in ensemble space, tile 16
    (36, 36, 32, 12, 12, 7.0),  # tile 32, 36 = 4 x 8 + 4: ragged runs
    (30, 28, 20, 10, 7, 6.0),   # k = 20: tile 24 with padding players
    (40, 40, 24, 4, 4, 9.0),    # both forms on one lattice (p from 2 to ~30)
]


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", ENS_CASES)
@pytest.mark.parametrize("run_len", [0, 1, 3, 8])
def test_ensemble_space_runs_match_oracle(gpu, nx, ny, k, nox, noy, d_cut, run_len):
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + 5 * k)
    f = _binary32_exact(f)
    got, _ = _mixed(gpu, f, ix, iy, yu, yv, d_cut, 1.05, run_len)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    assert norm_rel(got, ref) <= 5e-8
    assert norm_rel(ref, f) > 1e-6


def test_ensemble_space_warm_starts_take_fewer_sweeps(gpu):
    """256^2, 32 members, 16^2 observation points, d_cut = 32: every grid
    point in ensemble space (p ~ 100 > k); runs of 8 against one point per
    run."""
    nx = ny = 256
    k = 32
    f, ix, iy, yu, yv = _case(nx, ny, k, 16, 16, seed=8, steps=1)
    _, h8 = _mixed(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 8, hist=True)
    _, h1 = _mixed(gpu, f, ix, iy, yu, yv, 32.0, 1.05, 1, hist=True)
    assert h8.sum() == h1.sum() == nx * ny
    assert h8[31] == 0 and h1[31] == 0
    mean8 = (h8 * np.arange(32)).sum() / h8.sum()
    mean1 = (h1 * np.arange(32)).sum() / h1.sum()
    assert mean8 < 0.8 * mean1


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut,pipe", [
    (36, 20, 64, 3, 2, 9.0, 3),       # chunks of 3 runs, ragged last chunk and ragged runs
    (256, 256, 64, 8, 8, 32.0, 1024),  # the paper-scale lattice, 8 chunks
])
def test_pipelined_runs_equal_unpipelined(gpu, precision, nx, ny, k, nox, noy, d_cut, pipe):
    """letkf_set_run_pipeline: kernel J of the next chunk on the second
    stream beside the refinement of the current one gives the same state,
    bit for bit, as one chunk after another."""
    f, ix, iy, yu, yv = _case(nx, ny, k, nox, noy, seed=nx + 7 * k, steps=1)
    if precision == "mixed":
        f = _binary32_exact(f)
    prec = gpu.LBM_MIXED if precision == "mixed" else gpu.LBM_FP64
    out = []
    for p in (0, pipe):
        with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f) as e:
            e.set_run_length(8)
            e.set_run_pipeline(p)
            e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
            e.analyze(d_cut, 1.05)
            out.append(e.get_f())
            e.sync()
    assert np.array_equal(out[0], out[1])
    if nx <= 64:
        ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
        assert norm_rel(out[1], ref) <= (5e-8 if precision == "mixed" else 1e-12)


def test_run_pipeline_argument(gpu):
    with gpu.Ensemble(8, 8, 4, TAU0, CS, MU, gpu.LBM_MIXED) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.set_run_pipeline(-1)
        assert err.value.code == gpu.LBM_EINVAL
        e.set_run_pipeline(0)
        e.set_run_pipeline(4096)
