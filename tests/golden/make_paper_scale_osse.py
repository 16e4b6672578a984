"""Write the paper-scale OSSE reference: the first 1,000 steps (100 cycles)
of the 256^2 x 64-member LBM-LETKF experiment computed by the FP64 CPU
oracle (arXiv 2308.03972, Section 4.3: analysis every s = 10 steps, (u, v)
observed at 8 x 8 points with 10% noise, d_cut = 32, beta = 1.05).

This script calls only the oracle and the seeded input generators; the
GPU path is not involved. It writes tests/golden/paper_scale_osse.txt:
per cycle, the ensemble-mean velocity RMSE against the nature run before
and after the analysis, then the member-averaged energy spectrum of the
analysed ensemble after the last cycle.

    python tests/golden/make_paper_scale_osse.py [--cycles 100]

Run time: about 10 s per cycle on 8 cores.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_03972_gb300 import inputs  # noqa: E402  (seeded inputs only)

# The paper-scale configuration (lattice units; see the OSSE driver's
# defaults): 256^2, 64 members, 8 x 8 observation points, d_cut = 32,
# beta = 1.05, 10 steps per cycle, tau0 = 0.55, C_s = 0.2, rms Mach 0.05.
NX = NY = 256
K = 64
NOBS = 8
D_CUT = 32.0
BETA = 1.05
STEPS = 10
TAU0, CS, MU = 0.55, 0.2, 5e-4 * 0.001232
U_RMS = 0.05 / np.sqrt(3.0)
SIGMA = 0.1 * U_RMS
FORCE_AMP = 3.5e-6
SEEDS = {"nature": 1, "ensemble": 2, "forcing": 3, "noise": 4}


def mean_rmse(f, ut, vt):
    _, u, v = oracle.moments(f)
    return float(np.sqrt(np.mean((u.mean(2) - ut) ** 2 + (v.mean(2) - vt) ** 2)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cycles", type=int, default=100)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "paper_scale_osse.txt"))
    args = ap.parse_args()
    force = inputs.forcing_field(NX, NY, SEEDS["forcing"], FORCE_AMP, 3.0, 4.0)
    ix, iy = inputs.uniform_obs_points(NX, NY, NOBS, NOBS)
    tu, tv = inputs.random_velocity(NX, NY, SEEDS["nature"], U_RMS)
    nat = oracle.set_equilibrium(np.ones((NY, NX, 1)), tu[:, :, None], tv[:, :, None])
    eu, ev = inputs.ensemble_velocity(NX, NY, K, SEEDS["ensemble"], U_RMS, 0.1)
    f = oracle.set_equilibrium(np.ones_like(eu), eu, ev)
    rows = []
    t0 = time.time()
    for c in range(1, args.cycles + 1):
        nat = oracle.lbm_run(nat, force, TAU0, CS, MU, STEPS)
        _, u, v = oracle.moments(nat)
        ut, vt = u[:, :, 0], v[:, :, 0]
        nu, nv = inputs.obs_noise(SEEDS["noise"], c, len(ix))
        yu = ut[iy, ix] + SIGMA * nu
        yv = vt[iy, ix] + SIGMA * nv
        f = oracle.lbm_run(f, force, TAU0, CS, MU, STEPS)
        prior = mean_rmse(f, ut, vt)
        f = oracle.letkf_analyze(f, ix, iy, yu, yv, SIGMA, SIGMA, D_CUT, BETA)
        post = mean_rmse(f, ut, vt)
        rows.append((c, c * STEPS, prior, post))
        print("cycle %d step %d prior %.9e posterior %.9e (%.0f s)" % (c, c * STEPS, prior, post,
                                                                      time.time() - t0), flush=True)
    E = oracle.energy_spectrum(f)
    with open(args.out, "w") as fh:
        fh.write("# Paper-scale OSSE reference from the FP64 CPU oracle (arXiv 2308.03972,\n")
        fh.write("# Section 4.3): 256^2 lattice, 64 members, (u, v) at 8 x 8 points, 10% noise,\n")
        fh.write("# d_cut = 32, beta = 1.05, an analysis every 10 steps, %d cycles.\n" % args.cycles)
        fh.write("# Written by tests/golden/make_paper_scale_osse.py (oracle and seeded inputs only).\n")
        fh.write("# cycle  step  rmse_prior  rmse_posterior   (ensemble-mean velocity vs nature run)\n")
        for c, s, a, b in rows:
            fh.write("%d %d %.15e %.15e\n" % (c, s, a, b))
        fh.write("# spectrum after the last analysis: shell  E\n")
        for i, e in enumerate(E):
            fh.write("S %d %.15e\n" % (i, e))
    print("wrote", args.out)


if __name__ == "__main__":
    main()
