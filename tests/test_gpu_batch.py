"""Batches of independent experiments (lbm_batch_*): one persistent
cooperative launch advancing uneven ensembles, the launch-shape autotuner,
and DA cycles captured in a CUDA graph. Each is compared with the same
experiments run one call at a time through the single-context ABI (same
kernels, so bit-identical), and one experiment with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import TOL_FP64, U_RMS, norm_rel, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS
# Uneven experiments: lattice, members (k = 5 and 6 exercise 1 and 2 members
# per work item), observation lattice and radius.
EXPS = [(32, 24, 8, 4, 4, 6.0), (48, 40, 12, 6, 5, 9.0), (20, 20, 5, 4, 4, 5.0), (40, 32, 6, 5, 4, 7.0)]


def _states(precision_seed=0):
    out = []
    for i, (nx, ny, k, _, _, _) in enumerate(EXPS):
        f = turbulent_state(oracle, nx, ny, k, seed=10 + i + precision_seed, pert=0.2)
        force = inputs.forcing_field(nx, ny, seed=3 + i, amp=3.5e-6)
        out.append((f, force))
    return out


def _ensembles(gpu, prec, states):
    return [gpu.Ensemble(nx, ny, k, TAU0, CS, MU, prec, f0=f, force=force)
            for (nx, ny, k, _, _, _), (f, force) in zip(EXPS, states)]


def _obs(cycle):
    obs = []
    for i, (nx, ny, _, nox, noy, _) in enumerate(EXPS):
        ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
        tu, tv = inputs.random_velocity(nx, ny, 200 + i, U_RMS)
        nu, nv = inputs.obs_noise(4, cycle, len(ix))
        obs.append((ix, iy, tu[iy, ix] + SIGMA * nu, tv[iy, ix] + SIGMA * nv, SIGMA, SIGMA))
    return obs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_forecast_equals_single_context_forecasts(gpu, prec):
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    states = _states()
    ref = []
    for e in _ensembles(gpu, p, states):
        e.forecast(7)
        ref.append(e.get_f())
        e.close()
    ens = _ensembles(gpu, p, states)
    with gpu.Batch(ens) as b:
        b.forecast(3)
        b.forecast(4)
        b.sync()
    for e, r in zip(ens, ref):
        assert np.array_equal(e.get_f(), r)
        e.close()


def test_autotuned_shape_gives_the_same_forecast(gpu):
    states = _states()
    ens = _ensembles(gpu, gpu.LBM_MIXED, states)
    before = [e.get_f() for e in ens]
    with gpu.Batch(ens) as b:
        threads, blocks = b.autotune()
        assert threads in (128, 256, 512) and blocks >= 1
        for e, f0 in zip(ens, before):
            assert np.array_equal(e.get_f(), f0)  # tuning leaves the states alone
        b.forecast(5)
        b.sync()
    ref = _ensembles(gpu, gpu.LBM_MIXED, states)
    for e, r in zip(ens, ref):
        r.forecast(5)
        assert np.array_equal(e.get_f(), r.get_f())
        e.close()
        r.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_cycles_equal_single_context_cycles(gpu, prec):
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    states = _states()
    d_cut = [e[5] for e in EXPS]
    ncycles = 4
    ref = _ensembles(gpu, p, states)
    for c in range(1, ncycles + 1):
        for e, (ix, iy, yu, yv, su, sv), dc in zip(ref, _obs(c), d_cut):
            e.forecast(10)
            e.observe(ix, iy, yu, yv, su, sv)
            e.analyze(dc, 1.05)
    ens = _ensembles(gpu, p, states)
    with gpu.Batch(ens) as b:
        for c in range(1, ncycles + 1):
            b.cycle(10, _obs(c), d_cut, [1.05] * len(EXPS), use_graph=True)
        b.sync()
    for e, r in zip(ens, ref):
        assert np.array_equal(e.get_f(), r.get_f())
        e.close()
        r.close()


def test_graph_cycle_of_one_experiment_matches_oracle(gpu):
    nx, ny, k, nox, noy, d_cut = EXPS[0]
    f, force = _states()[0]
    ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
    ref = f
    e = gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f, force=force)
    with gpu.Batch([e]) as b:
        for c in range(1, 4):
            o = _obs(c)[0]
            ref = oracle.lbm_run(ref, force, TAU0, CS, MU, 10)
            ref = oracle.letkf_analyze(ref, ix, iy, o[2], o[3], SIGMA, SIGMA, d_cut, 1.05)
            b.cycle(10, [o], [d_cut], [1.05], use_graph=True)
        b.sync()
    assert norm_rel(e.get_f(), ref) <= TOL_FP64
    e.close()


def test_changed_plan_falls_back_and_still_matches(gpu):
    states = _states()
    d1 = [e[5] for e in EXPS]
    d2 = [x + 1.0 for x in d1]
    plan = [(1, d1), (2, d1), (3, d2), (4, d2), (5, d1)]
    ref = _ensembles(gpu, gpu.LBM_MIXED, states)
    for c, dc in plan:
        for e, (ix, iy, yu, yv, su, sv), d in zip(ref, _obs(c), dc):
            e.forecast(10)
            e.observe(ix, iy, yu, yv, su, sv)
            e.analyze(d, 1.05)
    ens = _ensembles(gpu, gpu.LBM_MIXED, states)
    with gpu.Batch(ens) as b:
        for c, dc in plan:
            b.cycle(10, _obs(c), dc, [1.05] * len(EXPS), use_graph=True)
        b.sync()
    for e, r in zip(ens, ref):
        assert np.array_equal(e.get_f(), r.get_f())
        e.close()
        r.close()


def test_batch_argument_errors(gpu):
    import torch

    states = _states()
    a = _ensembles(gpu, gpu.LBM_MIXED, states[:1])
    c = _ensembles(gpu, gpu.LBM_FP64, states[1:2])
    with pytest.raises(gpu.LbmError):
        gpu.Batch(a + c)  # mixed precisions
    with pytest.raises(gpu.LbmError):
        gpu.Batch(a + a)  # repeated context
    s = torch.cuda.Stream()
    nx, ny, k = EXPS[1][:3]
    other = gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_MIXED, f0=states[1][0], stream=s.cuda_stream)
    with pytest.raises(gpu.LbmError):
        gpu.Batch(a + [other])  # different streams
    with gpu.Batch(a) as b:
        with pytest.raises(gpu.LbmError):
            b.cycle(9, _obs(1)[:1], [6.0], [1.05], use_graph=True)  # odd nsteps with a graph
    for e in a + c + [other]:
        e.close()


def test_barrier_timeout_is_reported_and_the_batch_recovers(gpu):
    """Every grid-barrier wait runs out (one participant that never
    arrives, short spin limit): every block returns, lbm_batch_sync reports
    the timeout, and with normal barriers the batch works again."""
    states = _states()
    ens = _ensembles(gpu, gpu.LBM_MIXED, states)
    with gpu.Batch(ens) as b:
        b.set_barrier(20000, absent=1)
        b.forecast(3)  # stops at the first barrier, after one step
        with pytest.raises(gpu.LbmError) as err:
            b.sync()
        assert err.value.code == gpu.LBM_ECUDA and "timed out" in str(err.value)
        b.set_barrier(20000000, absent=0)
        b.forecast(2)
        b.sync()
    ref = _ensembles(gpu, gpu.LBM_MIXED, states)
    for e, r in zip(ens, ref):
        r.forecast(3)
        assert np.array_equal(e.get_f(), r.get_f())
        e.close()
        r.close()
    with gpu.Batch(_ensembles(gpu, gpu.LBM_MIXED, states[:1])) as b:
        with pytest.raises(gpu.LbmError):
            b.set_barrier(0)
        with pytest.raises(gpu.LbmError):
            b.set_barrier(1000, absent=2)


# The twelve experiments of the benchmark's batch leg: lattice side, members,
# observation lattice side, localisation radius.
TWELVE = [(128, 16, 8, 16.0), (128, 32, 16, 16.0), (128, 64, 8, 16.0), (128, 128, 8, 16.0),
          (256, 16, 16, 32.0), (256, 32, 8, 32.0), (256, 64, 8, 32.0), (256, 128, 16, 16.0),
          (512, 16, 32, 32.0), (512, 32, 16, 64.0), (512, 64, 8, 64.0), (512, 128, 32, 16.0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_twelve_experiments_match_oracle_at_sampled_points(gpu, prec):
    """One batch cycle (graph-captured) of the twelve uneven experiments;
    every experiment's analysis checked against the oracle's analysis of the
    same forecast state at sampled grid points."""
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    tol = TOL_FP64 if prec == "fp64" else 5e-8
    rng = np.random.default_rng(7)
    made, obs, dcs = [], [], []
    for i, (n, k, no, dc) in enumerate(TWELVE):
        u, v = inputs.ensemble_velocity(n, n, k, 50 + i, U_RMS, 0.2)
        force = inputs.forcing_field(n, n, seed=60 + i, amp=3.5e-6)
        ix, iy = inputs.uniform_obs_points(n, n, no, no)
        tu, tv = inputs.random_velocity(n, n, 70 + i, U_RMS)
        nu, nv = inputs.obs_noise(4, 1, len(ix))
        obs.append((ix, iy, tu[iy, ix] + SIGMA * nu, tv[iy, ix] + SIGMA * nv, SIGMA, SIGMA))
        made.append((n, k, u, v, force))
        dcs.append(dc)

    def build():
        out = []
        for n, k, u, v, force in made:
            e = gpu.Ensemble(n, n, k, TAU0, CS, MU, p, force=force)
            e.set_equilibrium(None, u, v)
            out.append(e)
        return out

    # The forecast state each analysis starts from (the batch forecast is
    # bit-identical to the cycle's, see the tests above).
    fc = build()
    with gpu.Batch(fc) as b:
        b.forecast(10)
        b.sync()
    ens = build()
    with gpu.Batch(ens) as b:
        b.cycle(10, obs, dcs, [1.05] * len(TWELVE), use_graph=True)
        b.sync()
    for i, (e, f) in enumerate(zip(ens, fc)):
        n = TWELVE[i][0]
        pts = np.unique(np.concatenate([rng.integers(0, n * n, 24), [0, n - 1, n * n - 1]])).astype(np.int32)
        f0 = f.get_f()
        ix, iy, yu, yv, su, sv = obs[i]
        ref = oracle.letkf_analyze(f0, ix, iy, yu, yv, su, sv, dcs[i], 1.05, points=pts)
        k = f0.shape[3]
        got = e.get_f().reshape(9, n * n, k)[:, pts]
        assert norm_rel(got, ref.reshape(9, n * n, k)[:, pts]) <= tol, "experiment %d" % i
        e.close()
        f.close()


def test_analysis_autotuner_keeps_states_and_cycles_match(gpu):
    """lbm_batch_autotune_analysis: run lengths and launch forms per size
    class timed on copies of the states (the states are unchanged), then
    batch cycles with the chosen run lengths and forms equal to
    single-context cycles with the same run lengths, bit for bit (same
    kernels)."""
    picks = [(128, 64, 8, 16.0), (128, 128, 8, 16.0), (256, 32, 8, 32.0), (128, 16, 8, 16.0)]
    made, obs = [], []
    for i, (n, k, no, dc) in enumerate(picks):
        u, v = inputs.ensemble_velocity(n, n, k, 80 + i, U_RMS, 0.2)
        force = inputs.forcing_field(n, n, seed=90 + i, amp=3.5e-6)
        ix, iy = inputs.uniform_obs_points(n, n, no, no)
        tu, tv = inputs.random_velocity(n, n, 100 + i, U_RMS)
        made.append((n, k, u, v, force))
        obs.append((ix, iy, tu, tv))
    dcs = [p[3] for p in picks]
    betas = [1.05] * len(picks)

    def cycle_obs(c):
        out = []
        for ix, iy, tu, tv in obs:
            nu, nv = inputs.obs_noise(4, c, len(ix))
            out.append((ix, iy, tu[iy, ix] + SIGMA * nu, tv[iy, ix] + SIGMA * nv, SIGMA, SIGMA))
        return out

    def build():
        out = []
        for n, k, u, v, force in made:
            e = gpu.Ensemble(n, n, k, TAU0, CS, MU, gpu.LBM_MIXED, force=force)
            e.set_equilibrium(None, u, v)
            out.append(e)
        return out

    ens = build()
    with gpu.Batch(ens) as b:
        b.forecast(10)
        for e, o in zip(ens, cycle_obs(1)):
            e.observe(*o)
        before = [e.get_f() for e in ens]
        rl = b.autotune_analysis(dcs, betas)
        for e, f0 in zip(ens, before):
            assert np.array_equal(e.get_f(), f0)
        # The first three take the run path; 16 members with 8 x 8 points
        # has ensemble-space points (its Jacobi kernel warm-starts along
        # runs): all four are tuned.
        assert all(r in (4, 8, 16, 32) for r in rl)
        # Launch form per experiment: either for the run-path classes; the
        # ensemble-space experiment keeps its own launches' default.
        assert all(m in (0, 1) for m in b.run_batched[:3])
        assert b.run_batched[3] == 1
        for c in (2, 3):
            b.cycle(10, cycle_obs(c), dcs, betas, use_graph=True)
        b.sync()
    ref = build()
    for e, r in zip(ref, rl):
        e.set_run_length(r)
        e.forecast(10)
    for c in (2, 3):
        for e, o, dc in zip(ref, cycle_obs(c), dcs):
            e.forecast(10)
            e.observe(*o)
            e.analyze(dc, 1.05)
    for e, r in zip(ens, ref):
        assert np.array_equal(e.get_f(), r.get_f())
        e.close()
        r.close()


def test_analysis_autotuner_needs_observations(gpu):
    ens = [gpu.Ensemble(16, 16, 8, TAU0, CS, MU, gpu.LBM_MIXED) for _ in range(2)]
    with gpu.Batch(ens) as b:
        with pytest.raises(gpu.LbmError) as err:
            b.autotune_analysis([4.0, 4.0], [1.05, 1.05])
        assert err.value.code == gpu.LBM_EINVAL
        with pytest.raises(ValueError):
            b.autotune_analysis([4.0], [1.05])
    for e in ens:
        e.close()


# Experiments on the run path (every grid point with p < k, unions of at
# most 32 scalars): the analysis launch form of the batch applies to them.
RUN_EXPS = [(64, 64, 64, 4, 4, 12.0), (48, 40, 48, 4, 4, 8.0)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_analysis_forms_agree(gpu, prec):
    """lbm_batch_set_analysis_form: the run analyses in the batched launch
    of kernel J and launched one experiment at a time give the same states,
    bit for bit, over uncaptured and graph-captured cycles."""
    p = gpu.LBM_FP64 if prec == "fp64" else gpu.LBM_MIXED
    dcs = [e[5] for e in RUN_EXPS]
    betas = [1.05] * len(RUN_EXPS)

    def build():
        out = []
        for i, (nx, ny, k, _, _, _) in enumerate(RUN_EXPS):
            u, v = inputs.ensemble_velocity(nx, ny, k, 60 + i, U_RMS, 0.2)
            force = inputs.forcing_field(nx, ny, seed=70 + i, amp=3.5e-6)
            e = gpu.Ensemble(nx, ny, k, TAU0, CS, MU, p, force=force)
            e.set_equilibrium(None, u, v)
            out.append(e)
        return out

    def obs(c):
        out = []
        for i, (nx, ny, _, nox, noy, _) in enumerate(RUN_EXPS):
            ix, iy = inputs.uniform_obs_points(nx, ny, nox, noy)
            tu, tv = inputs.random_velocity(nx, ny, 300 + i, U_RMS)
            nu, nv = inputs.obs_noise(6, c, len(ix))
            out.append((ix, iy, tu[iy, ix] + SIGMA * nu, tv[iy, ix] + SIGMA * nv, SIGMA, SIGMA))
        return out

    results = []
    for form in (1, 0):
        ens = build()
        with gpu.Batch(ens) as b:
            b.set_analysis_form([form] * len(ens))
            assert b.run_batched == [form] * len(ens)
            for c in (1, 2, 3):  # uncaptured, then captured and replayed
                b.cycle(4, obs(c), dcs, betas, use_graph=c > 1)
            b.sync()
            results.append([e.get_f() for e in ens])
        for e in ens:
            e.close()
    for a, b_ in zip(*results):
        assert np.array_equal(a, b_)


def test_batch_analysis_form_arguments(gpu):
    ens = [gpu.Ensemble(16, 16, 8, TAU0, CS, MU, gpu.LBM_MIXED) for _ in range(2)]
    with gpu.Batch(ens) as b:
        with pytest.raises(gpu.LbmError) as err:
            b.set_analysis_form([2, 0])
        assert err.value.code == gpu.LBM_EINVAL
        with pytest.raises(ValueError):
            b.set_analysis_form([1])
        b.set_analysis_form([0, 1])
    for e in ens:
        e.close()
