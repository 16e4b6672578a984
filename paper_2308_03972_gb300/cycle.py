"""Forecast-observe-analyse driver over the C ABI (arXiv 2308.03972, Section 3
workflow and Section 4.3 observing-system simulation experiment).

A ``Osse`` owns two contexts: the nature run (one member, FP64: the ground
truth) and the ensemble (k members, FP64 or mixed precision). One DA cycle is
    ensemble forecast of s steps -> observe -> LETKF analysis.
Observations are the nature run's velocity at the observation points plus
Gaussian noise; they are produced ahead of the cycles they feed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import binding, inputs


@dataclass
class OsseConfig:
    """One OSSE workload in lattice units. Defaults: 256^2 lattice, 64
    members, 8 x 8 (u, v) observation points, d_cut = 32, beta = 1.05, an
    analysis every 10 steps, tau0 = 0.55, C_s = 0.2, rms Mach 0.05."""
    nx: int = 256
    ny: int = 256
    members: int = 64
    nobs_x: int = 8
    nobs_y: int = 8
    d_cut: float = 32.0
    beta: float = 1.05
    steps_per_cycle: int = 10
    tau0: float = 0.55
    cs_smag: float = 0.2
    mu: float = 5e-4 * 0.001232       # Table 1 friction times the paper's dt
    mach: float = 0.05
    force_amp: float = 3.5e-6         # rms of F^i, lattice units per step
    force_kmin: float = 3.0
    force_kmax: float = 4.0
    noise: float = 0.1                # observation sigma / rms speed
    ens_pert: float = 0.1             # member perturbation / rms speed
    seeds: dict = field(default_factory=lambda: {"nature": 1, "ensemble": 2, "forcing": 3, "noise": 4})

    @property
    def u_rms(self) -> float:
        return self.mach / np.sqrt(3.0)

    @property
    def sigma(self) -> float:
        return self.noise * self.u_rms

    def name(self) -> str:
        return "lbm-letkf %dx%d k=%d obs=%dx%d d_cut=%g beta=%g s=%d" % (
            self.nx, self.ny, self.members, self.nobs_x, self.nobs_y, self.d_cut, self.beta,
            self.steps_per_cycle)


TINY = OsseConfig(nx=32, ny=32, members=8, nobs_x=4, nobs_y=4, d_cut=8.0)
PAPER_SCALE = OsseConfig()


class Osse:
    def __init__(self, cfg: OsseConfig, precision=binding.LBM_MIXED, stream="current"):
        self.cfg = cfg
        nx, ny, k = cfg.nx, cfg.ny, cfg.members
        self.force = inputs.forcing_field(nx, ny, cfg.seeds["forcing"], cfg.force_amp,
                                          cfg.force_kmin, cfg.force_kmax)
        self.ix, self.iy = inputs.uniform_obs_points(nx, ny, cfg.nobs_x, cfg.nobs_y)
        tu, tv = inputs.random_velocity(nx, ny, cfg.seeds["nature"], cfg.u_rms)
        eu, ev = inputs.ensemble_velocity(nx, ny, k, cfg.seeds["ensemble"], cfg.u_rms, cfg.ens_pert)
        self.nature = binding.Ensemble(nx, ny, 1, cfg.tau0, cfg.cs_smag, cfg.mu, binding.LBM_FP64,
                                       force=self.force, stream=stream)
        self.nature.set_equilibrium(None, tu[:, :, None].copy(), tv[:, :, None].copy())
        self.ens = binding.Ensemble(nx, ny, k, cfg.tau0, cfg.cs_smag, cfg.mu, precision,
                                    force=self.force, stream=stream)
        self.ens.set_equilibrium(None, eu, ev)
        self.cycle_index = 0
        self.truth_step = 0

    # -- truth ---------------------------------------------------------------
    def observations(self, ncycles: int):
        """Advance the nature run ncycles * s steps and return, per cycle, the
        observed (yo_u, yo_v) with noise, for the cycles that follow."""
        cfg = self.cfg
        out = []
        for c in range(ncycles):
            self.nature.forecast(cfg.steps_per_cycle)
            self.truth_step += cfg.steps_per_cycle
            u, v = self.nature.mean_velocity()
            cyc = self.truth_step // cfg.steps_per_cycle
            eu, ev = inputs.obs_noise(cfg.seeds["noise"], cyc, len(self.ix))
            out.append((u[self.iy, self.ix] + cfg.sigma * eu, v[self.iy, self.ix] + cfg.sigma * ev))
        return out

    def truth_velocity(self):
        return self.nature.mean_velocity()

    # -- one DA cycle ----------------------------------------------------------
    def cycle(self, yo):
        cfg = self.cfg
        self.ens.forecast(cfg.steps_per_cycle)
        self.ens.observe(self.ix, self.iy, yo[0], yo[1], cfg.sigma, cfg.sigma)
        self.ens.analyze(cfg.d_cut, cfg.beta)
        self.cycle_index += 1

    def rmse(self):
        """Velocity RMSE of the ensemble mean against the nature run (reduced
        on the device, lbm_velocity_rmse)."""
        return self.ens.velocity_rmse(self.nature)

    def close(self):
        self.ens.close()
        self.nature.close()
