"""Precision sweep at 256^2 (mixed-precision LBM state): members
k in {16, 32, 64, 128}, (u, v) observation lattices 8^2 .. 64^2 with 10%
noise, localisation radius d_cut = 32 and d_cut = the observation spacing,
and the Gram/b products in double-binary32 (FP64-class, the default), FP64,
binary32, TF32 and BF16 (eigensolve FP64-accurate in all). Every case is
checked against the FP64 oracle at sampled grid points; the error of each
case is printed as a table (run with -s to see it). Every case has n = min(k, p) <= 128, which the mixed path
holds; a case above it would have to be refused with LBM_EINVAL."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from paper_2308_03972_gb300.cycle import PAPER_SCALE as CFG

pytestmark = pytest.mark.gpu
NX = NY = 256
NSAMPLE = 16
BOUND = {"df32": 1e-6, "fp64": 1e-6, "fp32": 1e-6, "tf32": 2e-4, "bf16": 2e-3}  # of max |f^a|


def _max_local(no, d_cut, k):
    """Largest n = min(p, k) over the lattice: with the uniform observation
    lattice the local count repeats with the observation spacing, so one
    spacing cell of grid points covers every case."""
    ix, iy = inputs.uniform_obs_points(NX, NY, no, no)
    s = NX // no
    best = 0
    for y in range(s):
        for x in range(s):
            dx = np.abs(ix - x)
            dx = np.minimum(dx, NX - dx)
            dy = np.abs(iy - y)
            dy = np.minimum(dy, NY - dy)
            best = max(best, int(np.sum(np.sqrt(dx * dx + dy * dy) / d_cut < 2.0)))
    return min(2 * best, k)


def test_precision_sweep_256(gpu):
    rows = []
    force = inputs.forcing_field(NX, NY, CFG.seeds["forcing"], CFG.force_amp, CFG.force_kmin, CFG.force_kmax)
    tu, tv = inputs.random_velocity(NX, NY, CFG.seeds["nature"], CFG.u_rms)
    with gpu.Ensemble(NX, NY, 1, CFG.tau0, CFG.cs_smag, CFG.mu, gpu.LBM_FP64, force=force) as nat:
        nat.set_equilibrium(None, tu[:, :, None].copy(), tv[:, :, None].copy())
        nat.forecast(10)
        ut, vt = nat.mean_velocity()
        nat.sync()
    rng = np.random.default_rng(0)
    pts = np.sort(rng.choice(NX * NY, NSAMPLE, replace=False)).astype(np.int32)
    modes = (("df32", gpu.LBM_PROD_DF32), ("fp64", gpu.LBM_PROD_FP64), ("fp32", gpu.LBM_PROD_FP32),
             ("tf32", gpu.LBM_PROD_TF32), ("bf16", gpu.LBM_PROD_BF16))
    for k in (16, 32, 64, 128):
        eu, ev = inputs.ensemble_velocity(NX, NY, k, CFG.seeds["ensemble"], CFG.u_rms, CFG.ens_pert)
        with gpu.Ensemble(NX, NY, k, CFG.tau0, CFG.cs_smag, CFG.mu, gpu.LBM_MIXED, force=force) as e:
            e.set_equilibrium(None, eu, ev)
            e.forecast(10)
            f0 = e.get_f()
            for no in (8, 16, 32, 64):
                ix, iy = inputs.uniform_obs_points(NX, NY, no, no)
                nu, nv = inputs.obs_noise(CFG.seeds["noise"], 1, len(ix))
                yu = ut[iy, ix] + CFG.sigma * nu
                yv = vt[iy, ix] + CFG.sigma * nv
                for d_cut in sorted({32.0, float(NX // no)}):
                    n = _max_local(no, d_cut, k)
                    row = {"k": k, "obs": "%dx%d" % (no, no), "d_cut": d_cut, "n_max": n}
                    if n > 128:
                        e.set_f(f0)
                        e.observe(ix, iy, yu, yv, CFG.sigma, CFG.sigma)
                        with pytest.raises(gpu.LbmError) as err:
                            e.analyze(d_cut, CFG.beta)
                            e.sync()  # the device reports the size at the next sync
                        assert err.value.code == gpu.LBM_EINVAL
                        row["status"] = "refused: n > 128"
                        rows.append(row)
                        continue
                    ref = oracle.letkf_analyze(f0, ix, iy, yu, yv, CFG.sigma, CFG.sigma, d_cut, CFG.beta,
                                               points=pts)
                    y, x = pts // NX, pts % NX
                    ra = ref[:, y, x, :]
                    scale = np.max(np.abs(ra))
                    inc = np.max(np.abs(ra - f0[:, y, x, :]))
                    row["max_increment_rel"] = float(inc / scale)
                    for name, mode in modes:
                        e.set_f(f0)
                        e.set_products(mode)
                        e.observe(ix, iy, yu, yv, CFG.sigma, CFG.sigma)
                        e.analyze(d_cut, CFG.beta)
                        got = e.get_f()[:, y, x, :]
                        err_ = float(np.max(np.abs(got - ra)) / scale)
                        row[name] = err_
                        assert err_ <= BOUND[name], (row, name)
                    e.set_products(gpu.LBM_PROD_DF32)
                    row["status"] = "ok"
                    rows.append(row)
            e.sync()
    print()
    print("%4s %6s %6s %5s %10s %10s %10s %10s %10s %10s  %s" % ("k", "obs", "d_cut", "n", "increment", "df32",
                                                               "fp64", "fp32", "tf32", "bf16", "status"))
    for r in rows:
        if r["status"] == "ok":
            print("%4d %6s %6g %5d %10.2e %10.2e %10.2e %10.2e %10.2e %10.2e  ok" % (
                r["k"], r["obs"], r["d_cut"], r["n_max"], r["max_increment_rel"], r["df32"], r["fp64"],
                r["fp32"], r["tf32"], r["bf16"]))
        else:
            print("%4d %6s %6g %5d %s" % (r["k"], r["obs"], r["d_cut"], r["n_max"], r["status"]))
    out = os.environ.get("PRECISION_SWEEP_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump(rows, fh, indent=1)
