"""The first 1,000 steps (100 cycles) of the paper-scale observing-system
simulation (Section 4.3: 256^2 lattice, 64 members, (u, v) at 8 x 8 points
with 10% noise, d_cut = 32, beta = 1.05, an analysis every 10 steps)
against the FP64 CPU oracle's run stored in tests/golden/paper_scale_osse.txt
(written by tests/golden/make_paper_scale_osse.py from the oracle alone).

The observations and the truth are the oracle's nature run, recomputed here
on the CPU, so both sides assimilate the same data. Every cycle's
ensemble-mean velocity RMSE, before and after the analysis, must match the
oracle's to 1e-6 relative in FP64 mode and to 1% in mixed mode; the final
member-averaged energy spectrum must match shell by shell (1e-9 relative in
FP64 on shells above 1e-6 of the peak; 1% plus a floor of 1e-10 of the
total energy in mixed mode)."""
import os

import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from paper_2308_03972_gb300.cycle import PAPER_SCALE as CFG

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_scale_osse.txt")


def _golden():
    rows, spec = [], []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        if parts[0] == "S":
            spec.append(float(parts[2]))
        else:
            rows.append((int(parts[0]), int(parts[1]), float(parts[2]), float(parts[3])))
    return rows, np.array(spec)


@pytest.fixture(scope="module")
def osse():
    rows, spec = _golden()
    ncyc = len(rows)
    assert ncyc >= 100 and rows[-1][1] == 10 * ncyc
    nx, ny, k = CFG.nx, CFG.ny, CFG.members
    force = inputs.forcing_field(nx, ny, CFG.seeds["forcing"], CFG.force_amp, CFG.force_kmin, CFG.force_kmax)
    ix, iy = inputs.uniform_obs_points(nx, ny, CFG.nobs_x, CFG.nobs_y)
    tu, tv = inputs.random_velocity(nx, ny, CFG.seeds["nature"], CFG.u_rms)
    nat = oracle.set_equilibrium(np.ones((ny, nx, 1)), tu[:, :, None], tv[:, :, None])
    obs, truth = [], []
    for c in range(1, ncyc + 1):
        nat = oracle.lbm_run(nat, force, CFG.tau0, CFG.cs_smag, CFG.mu, CFG.steps_per_cycle)
        _, u, v = oracle.moments(nat)
        ut, vt = u[:, :, 0].copy(), v[:, :, 0].copy()
        nu, nv = inputs.obs_noise(CFG.seeds["noise"], c, len(ix))
        obs.append((ut[iy, ix] + CFG.sigma * nu, vt[iy, ix] + CFG.sigma * nv))
        truth.append((ut, vt))
    eu, ev = inputs.ensemble_velocity(nx, ny, k, CFG.seeds["ensemble"], CFG.u_rms, CFG.ens_pert)
    f0 = oracle.set_equilibrium(np.ones_like(eu), eu, ev)
    return {"rows": rows, "spec": spec, "force": force, "ix": ix, "iy": iy, "obs": obs, "truth": truth,
            "f0": f0}


def _run(gpu, ref, precision):
    nx, ny, k = CFG.nx, CFG.ny, CFG.members
    prior, post = [], []
    with gpu.Ensemble(nx, ny, k, CFG.tau0, CFG.cs_smag, CFG.mu, precision, f0=ref["f0"],
                      force=ref["force"]) as e:
        for (yu, yv), (ut, vt) in zip(ref["obs"], ref["truth"]):
            e.forecast(CFG.steps_per_cycle)
            um, vm = e.mean_velocity()
            prior.append(float(np.sqrt(np.mean((um - ut) ** 2 + (vm - vt) ** 2))))
            e.observe(ref["ix"], ref["iy"], yu, yv, CFG.sigma, CFG.sigma)
            e.analyze(CFG.d_cut, CFG.beta)
            um, vm = e.mean_velocity()
            post.append(float(np.sqrt(np.mean((um - ut) ** 2 + (vm - vt) ** 2))))
        E = e.energy_spectrum()
        e.sync()
    return np.array(prior), np.array(post), E


def test_fp64_first_1000_steps_match_oracle(gpu, osse):
    prior, post, E = _run(gpu, osse, gpu.LBM_FP64)
    ref_prior = np.array([r[2] for r in osse["rows"]])
    ref_post = np.array([r[3] for r in osse["rows"]])
    assert np.max(np.abs(prior / ref_prior - 1)) <= 1e-6
    assert np.max(np.abs(post / ref_post - 1)) <= 1e-6
    Er = osse["spec"]
    big = Er > 1e-6 * Er.max()
    assert np.max(np.abs(E[big] / Er[big] - 1)) <= 1e-9
    # The filter works: the error falls over the run.
    assert post[-1] < 0.5 * prior[0]


def test_mixed_first_1000_steps_within_one_percent(gpu, osse):
    prior, post, E = _run(gpu, osse, gpu.LBM_MIXED)
    ref_prior = np.array([r[2] for r in osse["rows"]])
    ref_post = np.array([r[3] for r in osse["rows"]])
    assert np.max(np.abs(prior / ref_prior - 1)) <= 1e-2
    assert np.max(np.abs(post / ref_post - 1)) <= 1e-2
    Er = osse["spec"]
    assert np.all(np.abs(E - Er) <= 1e-2 * Er + 1e-10 * Er.sum())
