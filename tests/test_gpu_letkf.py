"""Parity of the CUDA LETKF analysis and of the whole forecast-analysis
cycle with the FP64 oracle (arXiv 2308.03972, Section 3.2), called through
the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import TOL_FP64, U_RMS, norm_rel, osse_observations, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS


def _analysis_case(nx, ny, k, nobs_x, nobs_y, seed, steps=5):
    f = turbulent_state(oracle, nx, ny, k, seed=seed)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f = oracle.lbm_run(f, force, TAU0, CS, MU, steps)
    tu, tv = inputs.random_velocity(nx, ny, seed + 1000, U_RMS)
    ix, iy, yu, yv = osse_observations(nx, ny, nobs_x, nobs_y, 4, 1, tu, tv, SIGMA)
    return f, ix, iy, yu, yv


def _gpu_analysis(b, f, ix, iy, yu, yv, d_cut, beta, prec, sigma=SIGMA):
    _, ny, nx, k = f.shape
    with b.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f) as e:
        e.observe(ix, iy, yu, yv, sigma, sigma)
        e.analyze(d_cut, beta)
        out = e.get_f()
        e.sync()
    return out


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (24, 20, 8, 4, 4, 6.0),    # p >= k: ensemble-space form
    (30, 26, 8, 3, 2, 9.5),    # ragged lattice, ensemble-space form
    (24, 24, 40, 4, 4, 5.0),   # p < k: observation-space form
    (20, 20, 64, 2, 2, 7.0),   # observation-space form, two lanes per member
    (16, 16, 2, 4, 4, 4.0),    # smallest ensemble
])
def test_single_analysis_fp64_matches_oracle(gpu, nx, ny, k, nox, noy, d_cut):
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, nox, noy, seed=nx + k)
    beta = 1.05
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, beta, gpu.LBM_FP64)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, beta)
    assert norm_rel(got, ref) <= TOL_FP64
    # The analysis must actually change the ensemble.
    assert norm_rel(ref, f) > 1e-8


def test_no_observation_in_range_is_pure_inflation(gpu):
    f, ix, iy, yu, yv = _analysis_case(16, 16, 6, 2, 2, seed=9)
    # d_cut tiny: only cells on an observation point see it (r = 0).
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, 0.3, 1.1, gpu.LBM_FP64)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 0.3, 1.1)
    assert norm_rel(got, ref) <= TOL_FP64
    xbar = f.mean(axis=3, keepdims=True)
    mask = np.ones((16, 16), bool)
    mask[iy, ix] = False
    np.testing.assert_allclose(got[:, mask], (xbar + np.sqrt(1.1) * (f - xbar))[:, mask], rtol=0, atol=1e-15)


def test_observations_on_the_wrap_boundary(gpu):
    f, _, _, _, _ = _analysis_case(20, 18, 10, 2, 2, seed=11)
    ix = np.array([0, 19, 0, 19, 10], np.int32)
    iy = np.array([0, 0, 17, 17, 9], np.int32)
    yu = np.linspace(-0.02, 0.02, 5)
    yv = np.linspace(0.01, -0.01, 5)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, 4.0, 1.0, gpu.LBM_FP64)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 4.0, 1.0)
    assert norm_rel(got, ref) <= TOL_FP64


def test_full_size_analysis_sampled_points(gpu):
    """256^2 lattice, 64 members, 8 x 8 observation points, d_cut = 32: the
    configuration the benchmark times. Compared at sampled grid points."""
    nx = ny = 256
    k = 64
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, 8, 8, seed=21, steps=2)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, 32.0, 1.05, gpu.LBM_FP64)
    rng = np.random.default_rng(0)
    pts = np.unique(np.concatenate([rng.integers(0, nx * ny, 150),
                                    [0, nx - 1, nx * ny - 1, (ny - 1) * nx, 32 * nx + 32, 16 * nx + 48]]))
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 32.0, 1.05, points=pts.astype(np.int32))
    g = got.reshape(9, nx * ny, k)[:, pts]
    r = ref.reshape(9, nx * ny, k)[:, pts]
    assert norm_rel(g, r) <= TOL_FP64


def test_mixed_precision_analysis_close_to_oracle(gpu):
    f, ix, iy, yu, yv = _analysis_case(24, 24, 40, 4, 4, seed=31)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, 5.0, 1.05, gpu.LBM_MIXED)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 5.0, 1.05)
    assert norm_rel(got, ref) <= 1e-6


def test_argument_errors(gpu):
    f, ix, iy, yu, yv = _analysis_case(16, 16, 4, 2, 2, seed=2)
    with gpu.Ensemble(16, 16, 4, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        with pytest.raises(gpu.LbmError) as err:
            e.analyze(4.0, 1.0)  # no observation yet
        assert err.value.code == gpu.LBM_EINVAL
        with pytest.raises(gpu.LbmError):
            e.observe(np.array([16]), np.array([0]), [0.0], [0.0], SIGMA, SIGMA)
        with pytest.raises(gpu.LbmError):
            e.observe(ix, iy, yu, yv, 0.0, SIGMA)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        with pytest.raises(gpu.LbmError):
            e.analyze(-1.0, 1.0)
        e.analyze(4.0, 1.0)
        with pytest.raises(gpu.LbmError):
            e.analyze(4.0, 1.0)  # observation already consumed
        e.sync()
    with gpu.Ensemble(8, 8, 1, TAU0, CS, MU, gpu.LBM_FP64) as e:
        e.observe(np.array([1]), np.array([1]), [0.0], [0.0], SIGMA, SIGMA)
        with pytest.raises(gpu.LbmError):
            e.analyze(4.0, 1.0)  # one member


def test_oversized_local_problem_is_reported(gpu):
    """FP64 holds n = min(k, p) <= 64 and mixed precision n <= 128; a larger
    local problem is reported as LBM_EINVAL at the next sync."""
    # 80 members and 72 observation scalars in range: n = 72 > 64 (FP64).
    f, ix, iy, yu, yv = _analysis_case(24, 24, 80, 6, 6, seed=3)
    with gpu.Ensemble(24, 24, 80, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(100.0, 1.0)
        with pytest.raises(gpu.LbmError) as err:
            e.sync()
        assert err.value.code == gpu.LBM_EINVAL
    # 136 members and 288 observation scalars in range: n = 136 > 128.
    f, ix, iy, yu, yv = _analysis_case(24, 24, 136, 12, 12, seed=3, steps=1)
    for prec in (gpu.LBM_FP64, gpu.LBM_MIXED):
        with gpu.Ensemble(24, 24, 136, TAU0, CS, MU, prec, f0=f) as e:
            e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
            e.analyze(100.0, 1.0)
            with pytest.raises(gpu.LbmError) as err:
                e.sync()
            assert err.value.code == gpu.LBM_EINVAL


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (24, 24, 80, 6, 6, 100.0),    # observation space, n = 72
    (16, 16, 101, 8, 8, 100.0),   # ensemble space, n = k = 101 (odd)
    (20, 20, 128, 8, 8, 6.0),     # n = 112..128 over the grid, both forms, ragged
])
def test_local_problems_65_to_128_match_oracle(gpu, nx, ny, k, nox, noy, d_cut):
    """Mixed precision above n = 64: binary32 Jacobi with 64 round-robin
    pairs in shared memory, the refinement's A and A Y in global scratch."""
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, nox, noy, seed=70 + k)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, 1.05, gpu.LBM_MIXED)
    assert norm_rel(got, ref) <= 1e-6


@pytest.mark.parametrize("mode,bound", [("fp32", 1e-6), ("tf32", 2e-4), ("bf16", 2e-3)])
def test_reduced_gram_at_128_members(gpu, mode, bound):
    """The reduced-precision Gram pass at k = 128 (four passes of 32 output
    columns) in the ensemble-space form, against the FP64 oracle; bounds of
    max |f^a| as in the precision sweep."""
    nx, ny, k = 16, 16, 128
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, 8, 8, seed=5)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 100.0, 1.05)
    code = {"fp32": gpu.LBM_PROD_FP32, "tf32": gpu.LBM_PROD_TF32, "bf16": gpu.LBM_PROD_BF16}[mode]
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=f) as e:
        e.set_products(code)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(100.0, 1.05)
        got = e.get_f()
        e.sync()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= bound
    # The increment is far above the bound: the pass did change the state.
    assert np.max(np.abs(ref - f)) / np.max(np.abs(ref)) > 10 * bound


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (24, 24, 64, 6, 3, 100.0),   # observation space, n = 36
    (16, 16, 48, 8, 8, 100.0),   # ensemble space, n = k = 48
    (20, 20, 64, 5, 5, 7.0),     # observation space, n up to ~40, ragged local sets
])
def test_larger_local_problems_match_oracle(gpu, nx, ny, k, nox, noy, d_cut):
    """Local problems of 33..64 (two columns per lane in FP64; on the mixed
    path the 256-thread binary32 Jacobi and four warps per grid point in the
    refinement)."""
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, nox, noy, seed=70 + k)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, 1.05, gpu.LBM_FP64)
    assert norm_rel(got, ref) <= TOL_FP64
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, 1.05, gpu.LBM_MIXED)
    assert norm_rel(got, ref) <= 1e-6


def _osse(run_forecast, run_analysis, nature, steps, s, nobs, d_cut, beta, nx, ny, seed=4):
    """Cycle: forecast s steps, observe the nature run with noise, analyse."""
    for c in range(1, steps // s + 1):
        run_forecast(s)
        _, tu, tv = nature(c * s)
        ix, iy, yu, yv = osse_observations(nx, ny, nobs, nobs, seed, c, tu, tv, SIGMA)
        run_analysis(ix, iy, yu, yv, d_cut, beta)


def test_tiny_osse_cycle_fp64_and_mixed_match_oracle(gpu):
    """32^2 lattice, 8 members, 4 x 4 (u, v) observations, d_cut = 8,
    beta = 1.05, analysis every 10 steps for 200 steps."""
    nx = ny = 32
    k = 8
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    tu0, tv0 = inputs.random_velocity(nx, ny, 1, U_RMS)
    f_nat = oracle.set_equilibrium(np.ones((ny, nx, 1)), tu0[:, :, None], tv0[:, :, None])
    nature_states = {0: f_nat}
    for t in range(10, 201, 10):
        nature_states[t] = oracle.lbm_run(nature_states[t - 10], force, TAU0, CS, MU, 10)

    def nature(t):
        r, u, v = oracle.moments(nature_states[t])
        return r[:, :, 0], u[:, :, 0], v[:, :, 0]

    f0 = turbulent_state(oracle, nx, ny, k, seed=2)

    state = {"f": f0}

    def o_fc(n):
        state["f"] = oracle.lbm_run(state["f"], force, TAU0, CS, MU, n)

    def o_an(ix, iy, yu, yv, d_cut, beta):
        state["f"] = oracle.letkf_analyze(state["f"], ix, iy, yu, yv, SIGMA, SIGMA, d_cut, beta)

    _osse(o_fc, o_an, nature, 200, 10, 4, 8.0, 1.05, nx, ny)
    ref = state["f"]
    _, ur, vr = oracle.moments(ref)
    _, tu, tv = nature(200)
    rmse_ref = np.sqrt(np.mean((ur.mean(2) - tu) ** 2 + (vr.mean(2) - tv) ** 2))

    results = {}
    for prec in (gpu.LBM_FP64, gpu.LBM_MIXED):
        with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f0, force=force) as e:
            _osse(e.forecast, lambda ix, iy, yu, yv, d, b: (e.observe(ix, iy, yu, yv, SIGMA, SIGMA), e.analyze(d, b)),
                  nature, 200, 10, 4, 8.0, 1.05, nx, ny)
            got = e.get_f()
            _, ug, vg = e.moments_host()
            e.sync()
        rmse = np.sqrt(np.mean((ug.mean(2) - tu) ** 2 + (vg.mean(2) - tv) ** 2))
        results[prec] = (norm_rel(got, ref), abs(rmse / rmse_ref - 1))
    assert results[gpu.LBM_FP64][0] <= TOL_FP64
    assert results[gpu.LBM_FP64][1] <= 1e-6
    assert results[gpu.LBM_MIXED][1] <= 1e-2


def test_repeated_observe_calls_reuse_staging(gpu):
    """letkf_observe does not wait for the device: consecutive cycles with
    different observation sets give the oracle's result."""
    nx, ny, k = 20, 20, 6
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, 4, 4, seed=41)
    ref = f
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f) as e:
        for c in range(3):
            sel = slice(c, None)  # fewer points each cycle
            e.observe(ix[sel], iy[sel], yu[sel] * (1 + c), yv[sel], SIGMA, SIGMA)
            e.analyze(5.0, 1.05)
            ref = oracle.letkf_analyze(ref, ix[sel], iy[sel], yu[sel] * (1 + c), yv[sel], SIGMA, SIGMA, 5.0, 1.05)
        got = e.get_f()
    assert norm_rel(got, ref) <= TOL_FP64


@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [(24, 24, 40, 4, 4, 5.0), (24, 20, 8, 4, 4, 6.0)])
def test_mixed_analysis_stays_at_the_binary32_floor(gpu, nx, ny, k, nox, noy, d_cut):
    """On a state whose f - w is exact in binary32 (so both sides start from
    the same numbers), the mixed analysis stays within a few binary32 ulps of
    f - w (|f - w| <= 0.05) of the FP64 oracle: 5e-8 of max |f|."""
    from _helpers import W_REST

    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, nox, noy, seed=61 + k)
    w = np.asarray(W_REST)[:, None, None, None]
    f = ((f - w).astype(np.float32).astype(np.float64)) + w
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, 1.05, gpu.LBM_MIXED)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    assert norm_rel(got, ref) <= 5e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,k,nox,noy,d_cut", [
    (24, 20, 7, 4, 4, 6.0),     # odd k, ensemble space, one lane per column
    (20, 20, 33, 5, 5, 40.0),   # odd k, ensemble space, two columns per lane
    (20, 20, 45, 5, 5, 40.0),   # odd k in the 33..64 range
])
def test_odd_problem_sizes_match_oracle(gpu, prec, nx, ny, k, nox, noy, d_cut):
    """Odd n pads the round-robin with a player that never rotates; the
    real member of its pair must still be turned by the other rotations."""
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, nox, noy, seed=3 * k)
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, d_cut, 1.05, p)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
    assert norm_rel(got, ref) <= (TOL_FP64 if prec == "fp64" else 1e-6)


def test_mixed_analysis_over_many_odd_sized_chunks(gpu):
    """64^2 lattice, 100 members, 8 x 8 observation points all in range
    (d_cut = 100), so every local problem is the ensemble-space n = 100
    and a grid point needs 309,476 bytes of analysis scratch (basis, local
    list, FP64 Gram, refinement matrices). The 384 MiB budget then gives
    chunks of 1301 grid points (odd): four chunks alternate between the two
    scratch buffers, and the second buffer starts at an odd multiple of 4
    bytes unless the buffer size is rounded."""
    nx = ny = 64
    k = 100
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, 8, 8, seed=77, steps=2)
    got = _gpu_analysis(gpu, f, ix, iy, yu, yv, 100.0, 1.05, gpu.LBM_MIXED)
    rng = np.random.default_rng(5)
    pts = np.sort(rng.choice(nx * ny, 64, replace=False)).astype(np.int32)
    ref = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, 100.0, 1.05, points=pts)
    y, x = pts // nx, pts % nx
    assert norm_rel(got[:, y, x, :], ref[:, y, x, :]) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweep_histogram_counts_every_eigensolve(gpu, prec):
    """letkf_sweep_stats: one count per grid point with a non-empty local set,
    none at the sweep cap; off again, nothing is counted."""
    nx, ny, k = 24, 20, 8
    f, ix, iy, yu, yv = _analysis_case(nx, ny, k, 4, 4, seed=12)
    d_cut = 1.5  # support radius 3 < half the observation spacing: some points see nothing
    expected = sum(1 for y in range(ny) for x in range(nx)
                   if len(oracle.local_obs(nx, ny, x, y, ix, iy, SIGMA, SIGMA, d_cut)[0]) > 0)
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, p, f0=f) as e:
        e.sweep_stats(True)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        h = e.sweep_stats(False, read=True)
        e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
        e.analyze(d_cut, 1.05)
        h2 = e.sweep_stats(False, read=True)
        e.sync()
    assert 0 < expected < nx * ny
    assert int(h.sum()) == expected
    assert h[31] == 0 and h[0] == 0
    assert int(h2.sum()) == 0
