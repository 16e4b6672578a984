"""Benchmark of the LBM-LETKF forecast-analysis cycle on GB300.

One step = one DA cycle of the ensemble at the paper-scale workload
(256^2 lattice, 64 members, 8 x 8 (u, v) observation points, d_cut = 32,
beta = 1.05, 10 LBM steps per cycle): 10 fused LBM steps, the observation
operator and the LETKF analysis at all 65,536 grid points. The metric is
cycles/s; the primary line is the mixed-precision path, with the plain FP64
path measured on the same GPU alongside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun) every rank runs an independent replica (the cycle has
no exchange step on one lattice); value = cycles of all ranks / max time.
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LBM-LETKF cycles/s at 256^2 x 64 members (mixed precision; FP64 alongside)"
HBM_FALLBACK_GBS = 6800.0
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 (CUDA-core and tensor) nominal rate
FP32_LANES_PER_SM = 128       # binary32 FMA lanes per SM (4 sub-partitions x 32)
SM_MAX_MHZ_FALLBACK = 2070.0
L2_NOTE = "state larger than L2: 151 MB per buffer in FP32, 302 MB in FP64 (L2 = 129 MiB)"
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels at 256^2 x 64 (the summaries under profiles/; ncu flushes L2
# before each kernel). Set an entry to None when its kernel changes until it
# is captured again. Issue-slot utilisation of the two mixed-analysis
# kernels in the same capture.
ISSUE_ACTIVE = {"run_jacobi_kernel<28>": 0.748, "run_refine_kernel<28>": 0.585}
# Launches of one mixed analysis at 256^2 x 64 (runs of 8 grid points, one
# chunk of runs): binary32 copy of dY, split of the observation Gram, the
# Jacobi kernel and the refinement kernel.
MIXED_ANALYSIS_LAUNCHES = 4
NCU_TRAFFIC = {
    "analysis_mixed": 0.634112e6 + 167.438336e6 + 379.888384e6 + 117.160704e6,  # run kernels J + F
    "lbm_step_f32": 151.54816e6 + 97.796096e6,
    # FP64 run path: kernel J (as in the mixed path) + run_fp64_kernel.
    "analysis_fp64": 0.634112e6 + 167.438336e6 + 517.581568e6 + 251.356928e6,
}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    """Max of x over the ranks of the process group (x itself at world 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_per_cycle_max: float, world: int) -> float:
    """Whole-job cycles/s of `world` independent replicas timed by the slowest."""
    return world * 1000.0 / ms_per_cycle_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def local_obs_counts(cfg):
    """Number of local observation scalars at every grid point (host geometry:
    points with r / d_cut < 2 and a positive Gaspari-Cohn weight)."""
    from paper_2308_03972_gb300 import inputs

    ix, iy = inputs.uniform_obs_points(cfg.nx, cfg.ny, cfg.nobs_x, cfg.nobs_y)
    x = np.arange(cfg.nx)[None, :, None]
    y = np.arange(cfg.ny)[:, None, None]
    dx = np.abs(ix[None, None, :] - x)
    dx = np.minimum(dx, cfg.nx - dx)
    dy = np.abs(iy[None, None, :] - y)
    dy = np.minimum(dy, cfg.ny - dy)
    d = np.sqrt(dx * dx + dy * dy) / cfg.d_cut
    return 2 * (d < 2.0).sum(axis=2)


def analysis_flops(cfg, p):
    """Algorithmic FP64 flops of one analysis: per grid point with p local
    scalars and n = min(k, p) the eigensolve counts 9 n^3 (symmetric
    eigenvalues and vectors) and the dense products count 2 flops per
    multiply-add of their definition (observation-space form when p < k)."""
    k = cfg.members
    p = p.astype(np.float64)
    obs = p < k
    n = np.where(obs, p, k)
    eig = 9.0 * n ** 3
    prod_obs = 2 * (p * p + 2 * n * n + 9 * k * p + 2 * 9 * n * n + 9 * k * p)
    prod_ens = 2 * (k * k * p + k * p + 2 * k * k + k ** 3 + 9 * k * k)
    return float(np.sum(eig + np.where(obs, prod_obs, prod_ens)))


def measure(cfg, precision, steps, warmup, sample_clocks=False, gpu_index=0, run_length=8):
    import torch

    from paper_2308_03972_gb300 import binding
    from paper_2308_03972_gb300.cycle import Osse

    stream = torch.cuda.current_stream()
    osse = Osse(cfg, precision, stream=stream.cuda_stream)
    osse.ens.set_run_length(run_length)
    obs = osse.observations(warmup + steps)
    for c in range(warmup):
        osse.cycle(obs[c])
    osse.ens.sync()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_index) if sample_clocks else None
    if sampler:
        sampler.__enter__()
    try:
        torch.cuda.synchronize()
        start.record(stream)
        for c in range(steps):
            e = ev[c]
            yo = obs[warmup + c]
            e[0].record(stream)
            osse.ens.forecast(cfg.steps_per_cycle)
            e[1].record(stream)
            osse.ens.observe(osse.ix, osse.iy, yo[0], yo[1], cfg.sigma, cfg.sigma)
            e[2].record(stream)
            osse.ens.analyze(cfg.d_cut, cfg.beta)
            e[3].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
    finally:
        if sampler:
            sampler.__exit__()
    osse.ens.sync()
    # RMSE of the ensemble mean against the nature run at the same step.
    rmse = osse.rmse()
    # Jacobi sweeps per grid point, from one more (untimed) cycle.
    osse.ens.sweep_stats(True)
    osse.cycle(obs[-1])
    hist = osse.ens.sweep_stats(False, read=True)
    cum = np.cumsum(hist)
    sweeps = {"median": int(np.searchsorted(cum, cum[-1] / 2.0)), "max": int(np.nonzero(hist)[0].max()),
              "points": int(cum[-1])}
    # The nature run (one FP64 member) is the OSSE's truth, timed apart from
    # the ensemble cycle: one cycle's worth of steps, a few times.
    nat = []
    for _ in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        osse.nature.forecast(cfg.steps_per_cycle)
        b.record(stream)
        nat.append((a, b))
    torch.cuda.synchronize()
    nature_ms = statistics.median(a.elapsed_time(b) for a, b in nat)
    total_ms = start.elapsed_time(end)
    lbm = [e[0].elapsed_time(e[1]) / cfg.steps_per_cycle for e in ev]
    obs_ms = [e[1].elapsed_time(e[2]) for e in ev]
    ana = [e[2].elapsed_time(e[3]) for e in ev]
    osse.close()
    # Kernels per cycle: the LBM steps, observe + Gram, then the analysis
    # (mixed: MIXED_ANALYSIS_LAUNCHES; FP64 on runs: split Gram, kernel J,
    # the FP64 kernel; FP64 cold: one launch).
    if precision == binding.LBM_FP64:
        ana_launches = 3 if run_length > 0 else 1
    else:
        ana_launches = MIXED_ANALYSIS_LAUNCHES
    return {"ms_per_cycle": total_ms / steps, "lbm_step_ms": statistics.mean(lbm),
            "observe_ms": statistics.mean(obs_ms), "analysis_ms": statistics.mean(ana),
            "rmse": rmse, "clocks": sampler.summary() if sampler else None, "nature_ms": nature_ms,
            "sweeps": sweeps,
            "launches_per_cycle": cfg.steps_per_cycle + 2 + ana_launches}


def measure_e2e(cfg, precision, steps, warmup):
    """Public API with host buffers: each cycle copies its observations from
    host memory (pinned staging) and reads the ensemble-mean velocity back."""
    import torch

    from paper_2308_03972_gb300.cycle import Osse

    osse = Osse(cfg, precision)
    obs = osse.observations(warmup + steps)
    um = np.empty((cfg.ny, cfg.nx))
    vm = np.empty((cfg.ny, cfg.nx))
    for c in range(warmup):
        osse.cycle(obs[c])
        osse.ens.mean_velocity(um, vm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(steps):
        osse.cycle(obs[warmup + c])
        osse.ens.mean_velocity(um, vm)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    osse.close()
    npts = cfg.nobs_x * cfg.nobs_y
    return {"value": steps / dt, "unit": "cycles/s", "h2d_bytes_per_step": npts * (2 * 4 + 2 * 8),
            "d2h_bytes_per_step": 2 * cfg.nx * cfg.ny * 8}


def measure_graph(cfg, steps, warmup, run_length=8):
    """The same mixed-precision cycle captured in a CUDA graph: a batch of
    one experiment (lbm_batch_cycle: the forecast as one persistent launch,
    observe and analysis, replayed with only the observed values staged
    through pinned memory), device time per cycle."""
    import torch

    from paper_2308_03972_gb300 import binding
    from paper_2308_03972_gb300.cycle import Osse

    stream = torch.cuda.current_stream()
    osse = Osse(cfg, binding.LBM_MIXED, stream=stream.cuda_stream)
    osse.ens.set_run_length(run_length)
    obs = osse.observations(warmup + steps + 2)

    def one(c):
        yo = obs[c]
        return [(osse.ix, osse.iy, yo[0], yo[1], cfg.sigma, cfg.sigma)]

    with binding.Batch([osse.ens]) as b:
        for c in range(2 + warmup):  # uncaptured, captured, then warm replays
            b.cycle(cfg.steps_per_cycle, one(c), [cfg.d_cut], [cfg.beta], use_graph=True)
        b.sync()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c in range(steps):
            b.cycle(cfg.steps_per_cycle, one(2 + warmup + c), [cfg.d_cut], [cfg.beta], use_graph=True)
        z.record(stream)
        b.sync()
    ms = a.elapsed_time(z) / steps
    osse.close()
    return {"value": 1000.0 / ms, "unit": "cycles/s", "ms_per_step": ms,
            "note": "the same cycle as value, captured in a CUDA graph through lbm_batch_cycle (one experiment)"}


def measure_osse(cfg, precision, cycles=1000, every=10):
    """The paper's observing-system simulation at the paper scale (Section
    4.3): `cycles` forecast-analysis cycles (10 steps each; 1,000 cycles =
    10,000 steps), the ensemble-mean velocity RMSE against the nature run
    every `every` cycles, and its end against the observation-noise RMS
    sqrt(2) sigma."""
    import torch

    from paper_2308_03972_gb300.cycle import Osse

    osse = Osse(cfg, precision)
    curve = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(cycles):
        # The nature run advances with the ensemble, so that every point of
        # the curve compares the two at the same step.
        obs = osse.observations(1)
        osse.cycle(obs[0])
        if (c + 1) % every == 0:
            curve.append(osse.rmse())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    osse.close()
    noise = cfg.sigma * np.sqrt(2.0)
    return {"cycles": cycles, "steps": cycles * cfg.steps_per_cycle, "every_cycles": every,
            "rmse_curve": curve, "rmse_final": curve[-1], "rmse_min": min(curve),
            "obs_noise_rms": noise, "final_below_obs_noise": bool(curve[-1] < noise),
            "wall_s": dt, "wall_includes": "nature run (FP64, one member) and its observation read-back per cycle"}


def measure_adjoint(cfg, reps=3, nsteps=200, ckpt=20):
    """Gradient of a 200-step windowed (u, v) misfit for a batch of 64
    initial states on the 256^2 lattice in binary32: observations of the
    nature run at 16 x 16 points after every 10 steps (10% noise),
    checkpoints every 20 steps, gradient left on the device."""
    import torch

    from paper_2308_03972_gb300 import binding, inputs

    every, side = 10, 16
    nx, ny, k = cfg.nx, cfg.ny, cfg.members
    force = inputs.forcing_field(nx, ny, cfg.seeds["forcing"], cfg.force_amp, cfg.force_kmin, cfg.force_kmax)
    ix, iy = inputs.uniform_obs_points(nx, ny, side, side)
    tu, tv = inputs.random_velocity(nx, ny, cfg.seeds["nature"], cfg.u_rms)
    nat = binding.Ensemble(nx, ny, 1, cfg.tau0, cfg.cs_smag, cfg.mu, binding.LBM_FP64, force=force)
    nat.set_equilibrium(None, tu[:, :, None].copy(), tv[:, :, None].copy())
    yu, yv = [], []
    for t in range(every, nsteps + 1, every):
        nat.forecast(every)
        u, v = nat.mean_velocity()
        nu, nv = inputs.obs_noise(cfg.seeds["noise"], t, len(ix))
        yu.append(u[iy, ix] + cfg.sigma * nu)
        yv.append(v[iy, ix] + cfg.sigma * nv)
    nat.close()
    win = binding.Window(nsteps, every, ix, iy, np.array(yu), np.array(yv), cfg.sigma, cfg.sigma, ckpt)
    eu, ev = inputs.ensemble_velocity(nx, ny, k, cfg.seeds["ensemble"], cfg.u_rms, cfg.ens_pert)
    ens = binding.Ensemble(nx, ny, k, cfg.tau0, cfg.cs_smag, cfg.mu, binding.LBM_MIXED, force=force)
    ens.set_equilibrium(None, eu, ev)
    grad = torch.empty((9, ny, nx, k), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    binding.lbm_misfit_gradient(ens.ctx, win, k, grad_f0=grad)  # warm-up
    times, ftimes = [], []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        binding.lbm_misfit_gradient(ens.ctx, win, k, grad_f0=grad)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        a.record(stream)
        ens.misfit(win)
        b.record(stream)
        torch.cuda.synchronize()
        ftimes.append(a.elapsed_time(b))
    ens.close()
    ms = statistics.median(times)
    fms = statistics.median(ftimes)
    upd = nx * ny * k
    # Algorithmic HBM bytes: forward 200 steps and recomputation of 180 (read
    # + write 9 binary32 values), 200 adjoint steps (read f_t and lambda,
    # write lambda), the checkpoint copies, and the FP64 gradient write.
    nrec = nsteps - nsteps // ckpt
    byts = (nsteps + nrec) * 72 * upd + nsteps * 108 * upd + (nsteps // ckpt) * 72 * upd + 9 * 12 * upd
    return {"workload": "256x256 x 64 initial states, %d-step window, (u,v) misfit at 16x16 points every "
                        "10 steps, checkpoints every %d steps, binary32 forecast and adjoint" % (nsteps, ckpt),
            "ms_per_window_gradient": ms, "ms_per_window_misfit_only": fms,
            "gradients_per_s": 1000.0 / ms, "algorithmic_bytes": byts,
            "achieved_gbs": byts / (ms * 1e6)}


def measure_sweep(cfg, reps=2, only=None):
    """Analysis time of the precision sweep at 256^2 (binary32 LBM state):
    k in {16, 32, 64, 128}, observation lattices 8^2 .. 64^2, d_cut = 32 and
    d_cut = the observation spacing, Gram/b products double-binary32 / FP64 /
    binary32 / TF32 / BF16. Every case fits the mixed path (n = min(k, p) <= 128); one above
    it would be listed as refused. only = (k, obs side, d_cut) restricts the
    sweep to that case."""
    import torch

    from paper_2308_03972_gb300 import binding, inputs

    nx, ny = cfg.nx, cfg.ny
    force = inputs.forcing_field(nx, ny, cfg.seeds["forcing"], cfg.force_amp, cfg.force_kmin, cfg.force_kmax)
    tu, tv = inputs.random_velocity(nx, ny, cfg.seeds["nature"], cfg.u_rms)
    stream = torch.cuda.current_stream()
    modes = (("df32", binding.LBM_PROD_DF32), ("fp64", binding.LBM_PROD_FP64), ("fp32", binding.LBM_PROD_FP32),
             ("tf32", binding.LBM_PROD_TF32), ("bf16", binding.LBM_PROD_BF16))
    out = []
    for k in (16, 32, 64, 128):
        if only and k != only[0]:
            continue
        eu, ev = inputs.ensemble_velocity(nx, ny, k, cfg.seeds["ensemble"], cfg.u_rms, cfg.ens_pert)
        ens = binding.Ensemble(nx, ny, k, cfg.tau0, cfg.cs_smag, cfg.mu, binding.LBM_MIXED, force=force)
        ens.set_equilibrium(None, eu, ev)
        ens.forecast(10)
        for no in (8, 16, 32, 64):
            ix, iy = inputs.uniform_obs_points(nx, ny, no, no)
            nu, nv = inputs.obs_noise(cfg.seeds["noise"], 1, len(ix))
            yu, yv = tu[iy, ix] + cfg.sigma * nu, tv[iy, ix] + cfg.sigma * nv
            for d_cut in sorted({32.0, float(nx // no)}):
                if only and (no != only[1] or d_cut != only[2]):
                    continue
                row = {"k": k, "obs": "%dx%d" % (no, no), "d_cut": d_cut}
                for name, mode in modes:
                    ens.set_products(mode)
                    ts = []
                    try:
                        for r in range(reps + 1):
                            ens.observe(ix, iy, yu, yv, cfg.sigma, cfg.sigma)
                            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            a.record(stream)
                            ens.analyze(d_cut, cfg.beta)
                            b.record(stream)
                            ens.sync()
                            if r:
                                ts.append(a.elapsed_time(b))
                        row[name + "_ms"] = statistics.median(ts)
                    except binding.LbmError as err:
                        row["status"] = "refused: " + str(err).split(": ", 1)[-1]
                        break
                out.append(row)
        ens.close()
    return out


# Twelve uneven DA experiments (lattice, members, observation lattice side,
# localisation radius), all within local problems of n <= 64.
BATCH_EXPERIMENTS = [
    (128, 16, 8, 16.0), (128, 32, 16, 16.0), (128, 64, 8, 16.0), (128, 128, 8, 16.0),
    (256, 16, 16, 32.0), (256, 32, 8, 32.0), (256, 64, 8, 32.0), (256, 128, 16, 16.0),
    (512, 16, 32, 32.0), (512, 32, 16, 64.0), (512, 64, 8, 64.0), (512, 128, 32, 16.0),
]


def measure_batch(cfg, cycles=3):
    """Twelve independent experiments (lattices 128^2..512^2, k 16..128,
    observations 8^2..32^2, d_cut 16..64), binary32 LBM, s = 10: one batch
    cycle = persistent forecast of all + observe + analysis of all. Timed
    as a captured CUDA graph and as plain per-context calls."""
    import torch

    from paper_2308_03972_gb300 import binding, inputs

    stream = torch.cuda.current_stream()
    ens, obs_pos, truths, dcs = [], [], [], []
    for i, (n, k, no, dc) in enumerate(BATCH_EXPERIMENTS):
        force = inputs.forcing_field(n, n, cfg.seeds["forcing"] + i, cfg.force_amp, cfg.force_kmin, cfg.force_kmax)
        eu, ev = inputs.ensemble_velocity(n, n, k, cfg.seeds["ensemble"] + i, cfg.u_rms, cfg.ens_pert)
        e = binding.Ensemble(n, n, k, cfg.tau0, cfg.cs_smag, cfg.mu, binding.LBM_MIXED, force=force)
        e.set_equilibrium(None, eu, ev)
        ens.append(e)
        obs_pos.append(inputs.uniform_obs_points(n, n, no, no))
        truths.append(inputs.random_velocity(n, n, cfg.seeds["nature"] + i, cfg.u_rms))
        dcs.append(dc)

    def obs(c):
        out = []
        for (ix, iy), (tu, tv) in zip(obs_pos, truths):
            nu, nv = inputs.obs_noise(cfg.seeds["noise"], c, len(ix))
            out.append((ix, iy, tu[iy, ix] + cfg.sigma * nu, tv[iy, ix] + cfg.sigma * nv, cfg.sigma, cfg.sigma))
        return out

    betas = [cfg.beta] * len(ens)
    res = {"experiments": [{"n": n, "k": k, "obs": "%dx%d" % (no, no), "d_cut": dc}
                           for n, k, no, dc in BATCH_EXPERIMENTS]}
    with binding.Batch(ens) as b:
        res["autotuned_threads"], res["autotuned_blocks"] = b.autotune()
        # One plain cycle, then the run length per size class of the batched
        # analyses, tuned on the next observations (states unchanged).
        c = 1
        b.cycle(10, obs(c), dcs, betas, use_graph=False)
        c += 1
        b.forecast(10)
        for e, o in zip(ens, obs(c)):
            e.observe(*o)
        c += 1
        res["autotuned_run_len"] = b.autotune_analysis(dcs, betas)
        res["autotuned_run_batched"] = b.run_batched
        for _ in range(2):  # uncaptured first cycle, then capture
            b.cycle(10, obs(c), dcs, betas, use_graph=True)
            c += 1
        b.sync()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(cycles):
            b.cycle(10, obs(c), dcs, betas, use_graph=True)
            c += 1
        z.record(stream)
        b.sync()
        graph_ms = a.elapsed_time(z) / cycles
        a.record(stream)
        b.forecast(10)
        z.record(stream)
        b.sync()
        res["persistent_forecast_ms"] = a.elapsed_time(z)
    # The same cycles through the single-context calls.
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(cycles):
        for e, (ix, iy, yu, yv, su, sv), dc in zip(ens, obs(c), dcs):
            e.forecast(10)
            e.observe(ix, iy, yu, yv, su, sv)
            e.analyze(dc, cfg.beta)
        c += 1
    z.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(z) / cycles
    a.record(stream)
    for e in ens:
        e.forecast(10)
    z.record(stream)
    torch.cuda.synchronize()
    res["per_context_forecast_ms"] = a.elapsed_time(z)
    for e in ens:
        e.close()
    upd = sum(n * n * k for n, k, _, _ in BATCH_EXPERIMENTS) * 10
    res.update({"ms_per_batch_cycle_graph": graph_ms, "ms_per_batch_cycle_plain": plain_ms,
                "experiment_cycles_per_s": len(BATCH_EXPERIMENTS) * 1000.0 / graph_ms,
                "forecast_gbs_persistent": upd * 72 / (res["persistent_forecast_ms"] * 1e6)})
    return res


def _oracle_inputs(cfg):
    import oracle
    from paper_2308_03972_gb300 import inputs

    nx, ny, k = cfg.nx, cfg.ny, cfg.members
    u, v = inputs.ensemble_velocity(nx, ny, k, cfg.seeds["ensemble"], cfg.u_rms, cfg.ens_pert)
    f = oracle.set_equilibrium(np.ones_like(u), u, v)
    force = inputs.forcing_field(nx, ny, cfg.seeds["forcing"], cfg.force_amp, cfg.force_kmin, cfg.force_kmax)
    ix, iy = inputs.uniform_obs_points(nx, ny, cfg.nobs_x, cfg.nobs_y)
    tu, tv = inputs.random_velocity(nx, ny, cfg.seeds["nature"], cfg.u_rms)
    eu, ev = inputs.obs_noise(cfg.seeds["noise"], 1, len(ix))
    return f, force, ix, iy, tu[iy, ix] + cfg.sigma * eu, tv[iy, ix] + cfg.sigma * ev


def oracle_cycle(cfg, f, force, ix, iy, yu, yv):
    """One full FP64 oracle cycle: s LBM steps of the ensemble and the LETKF
    analysis at every grid point (observation operator included)."""
    import oracle

    f = oracle.lbm_run(f, force, cfg.tau0, cfg.cs_smag, cfg.mu, cfg.steps_per_cycle)
    return oracle.letkf_analyze(f, ix, iy, yu, yv, cfg.sigma, cfg.sigma, cfg.d_cut, cfg.beta)


def oracle_baseline(cfg, steps_timed=5, analyses_timed=3, st_points=2048):
    """The FP64 oracle on the host cores (about 20 s on 16 cores):
      * all cores: median of `steps_timed` LBM steps and of `analyses_timed`
        full analyses at the paper scale; cycle = s steps + one analysis;
      * one thread: one LBM step and the analysis at `st_points` sampled grid
        points, extrapolated to the whole lattice (labelled);
      * the tiny configuration (32^2, k = 8, 4 x 4 points, d_cut = 8,
        200 steps, 20 analyses), timed whole on all cores."""
    import oracle
    from paper_2308_03972_gb300.cycle import TINY

    cores = oracle.num_threads()
    f, force, ix, iy, yu, yv = _oracle_inputs(cfg)
    ts = []
    for _ in range(steps_timed):
        t0 = time.perf_counter()
        f1 = oracle.lbm_step(f, force, cfg.tau0, cfg.cs_smag, cfg.mu)
        ts.append(time.perf_counter() - t0)
    ta = []
    for _ in range(analyses_timed):
        t0 = time.perf_counter()
        oracle.letkf_analyze(f1, ix, iy, yu, yv, cfg.sigma, cfg.sigma, cfg.d_cut, cfg.beta)
        ta.append(time.perf_counter() - t0)
    t_step, t_ana = statistics.median(ts), statistics.median(ta)
    t_cycle = cfg.steps_per_cycle * t_step + t_ana
    # One thread, bounded sample.
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.lbm_step(f, force, cfg.tau0, cfg.cs_smag, cfg.mu)
        st_step = time.perf_counter() - t0
        rng = np.random.default_rng(0)
        pts = np.sort(rng.choice(cfg.nx * cfg.ny, size=st_points, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.letkf_analyze(f1, ix, iy, yu, yv, cfg.sigma, cfg.sigma, cfg.d_cut, cfg.beta, points=pts)
        st_ana = (time.perf_counter() - t0) * (cfg.nx * cfg.ny) / st_points
    finally:
        oracle.set_num_threads(cores)
    st_cycle = cfg.steps_per_cycle * st_step + st_ana
    # The tiny configuration, whole.
    ft, forcet, ixt, iyt, _, _ = _oracle_inputs(TINY)
    from paper_2308_03972_gb300 import inputs
    tut, tvt = inputs.random_velocity(TINY.nx, TINY.ny, TINY.seeds["nature"], TINY.u_rms)
    t0 = time.perf_counter()
    for c in range(1, 21):
        nu, nv = inputs.obs_noise(TINY.seeds["noise"], c, len(ixt))
        ft = oracle_cycle(TINY, ft, forcet, ixt, iyt, tut[iyt, ixt] + TINY.sigma * nu, tvt[iyt, ixt] + TINY.sigma * nv)
    t_tiny = time.perf_counter() - t0
    return {"value": 1.0 / t_cycle, "unit": "cycles/s", "cores": cores, "kind": "oracle",
            "sample": "FP64 C oracle (OpenMP, %d threads) at 256^2 x 64: median of %d LBM steps and of %d "
                      "full analyses (all 65536 grid points); cycle = 10 steps + 1 analysis"
                      % (cores, steps_timed, analyses_timed),
            "lbm_step_s": t_step, "analysis_s": t_ana,
            "single_thread": {"value": 1.0 / st_cycle, "unit": "cycles/s", "cores": 1,
                              "sample": "1 LBM step + analysis at %d of %d grid points, extrapolated"
                                        % (st_points, cfg.nx * cfg.ny),
                              "lbm_step_s": st_step, "analysis_s": st_ana},
            "tiny_whole": {"workload": TINY.name(), "seconds": t_tiny, "cycles": 20,
                           "cycles_per_s": 20.0 / t_tiny, "cores": cores}}


def run_reference(args, cfg):
    """The reference arm: the FP64 oracle as it stands on the host cores.
    Each step is one full paper-scale cycle (10 LBM steps of the 64-member
    ensemble + the LETKF analysis at all 65536 grid points), so steps x
    ms_per_step is the time that actually ran."""
    import oracle

    rank, world, _ = _dist()
    if rank != 0:
        return
    f, force, ix, iy, yu, yv = _oracle_inputs(cfg)
    for _ in range(args.warmup):
        f = oracle_cycle(cfg, f, force, ix, iy, yu, yv)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle_cycle(cfg, f, force, ix, iy, yu, yv)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cycles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg.name(), "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "cycles/s", "cores": cores, "kind": "oracle",
                             "sample": "full cycles of the workload (10 LBM steps + analysis at every grid "
                                       "point), FP64 C oracle, OpenMP %d threads; observations of one "
                                       "cycle reused" % cores},
            "e2e": {"value": value, "unit": "cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--run-length", type=int, default=8,
                    help="grid points per run of the analysis, both precisions (0: one grid point per warp, "
                         "cold-started)")
    ap.add_argument("--window", type=int, default=200, help="adjoint window steps (--case adjoint)")
    ap.add_argument("--checkpoint", type=int, default=20, help="adjoint checkpoint spacing (--case adjoint)")
    ap.add_argument("--sweep-only", default=None,
                    help="k:obs:d_cut, one case of the precision sweep (--case sweep)")
    ap.add_argument("--case", default="all", choices=["all", "cycle", "adjoint", "sweep", "batch", "osse"],
                    help="cycle: the headline line without the adjoint, batch and OSSE legs; adjoint: only "
                         "the adjoint-window leg; sweep: precision-sweep timings; batch: twelve uneven "
                         "experiments; osse: the 10,000-step OSSE in both precisions")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    from paper_2308_03972_gb300.cycle import PAPER_SCALE
    cfg = PAPER_SCALE
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_2308_03972_gb300 import binding, build

    build.build()
    binding.load()

    barrier_max = lambda x: reduce_max(x, world)  # noqa: E731
    if args.case == "batch":
        res = measure_batch(cfg)
        if rank == 0:
            print(json.dumps({"case": "batch", **res}))
        return
    if args.case == "sweep":
        only = None
        if args.sweep_only:
            kk, no, dc = args.sweep_only.split(":")
            only = (int(kk), int(no), float(dc))
        for row in measure_sweep(cfg, only=only):
            if rank == 0:
                print(json.dumps({"case": "sweep", **row}))
        return
    if args.case == "osse":
        res = {"case": "osse", "workload": cfg.name(),
               "mixed": measure_osse(cfg, binding.LBM_MIXED), "fp64": measure_osse(cfg, binding.LBM_FP64)}
        if rank == 0:
            print(json.dumps(res))
        return
    if args.case == "adjoint":
        adj = measure_adjoint(cfg, reps=args.steps, nsteps=args.window, ckpt=args.checkpoint)
        if rank == 0:
            print(json.dumps({"case": "adjoint", **adj}))
        return

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    mixed = measure(cfg, binding.LBM_MIXED, args.steps, args.warmup, sample_clocks=(rank == 0), gpu_index=local,
                    run_length=args.run_length)
    ms = barrier_max(mixed["ms_per_cycle"])
    fp64 = measure(cfg, binding.LBM_FP64, max(3, args.steps // 3), args.warmup, run_length=args.run_length)
    ms64 = barrier_max(fp64["ms_per_cycle"])
    e2e = measure_e2e(cfg, binding.LBM_MIXED, args.steps, args.warmup)
    graph = measure_graph(cfg, args.steps, args.warmup, run_length=args.run_length)
    e2e_val = barrier_max(1.0 / e2e["value"])

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    sm_mhz = peaks.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    # Binary32 peak derived from the unit counts and the maximum SM clock:
    # SMs x 128 FMA lanes x 2 flops x clock.
    fp32_gflops = nsm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e-3
    p = local_obs_counts(cfg)
    flops = analysis_flops(cfg, p)
    ncell = cfg.nx * cfg.ny * cfg.members
    lbm_bytes32 = 2 * 9 * 4 * ncell
    lbm_bytes64 = 2 * 9 * 8 * ncell
    ana_bytes32 = 2 * 9 * 4 * ncell  # f read and written once per analysis (binary32)
    ana_bytes64 = 2 * 9 * 8 * ncell
    kern = {
        "lbm_step_f32": {"ms": mixed["lbm_step_ms"], "launches_per_cycle": cfg.steps_per_cycle,
                         "bound": "hbm", "achieved_gbs": lbm_bytes32 / (mixed["lbm_step_ms"] * 1e6),
                         "peak_gbs": hbm, "frac": lbm_bytes32 / (mixed["lbm_step_ms"] * 1e6) / hbm},
        "analysis_mixed": {"ms": mixed["analysis_ms"],
                           "launches_per_cycle": mixed["launches_per_cycle"] - cfg.steps_per_cycle - 2,
                           "bound": "alu (binary32)",
                           "achieved_gflops": flops / (mixed["analysis_ms"] * 1e6),
                           "peak_gflops": fp32_gflops,
                           "frac": flops / (mixed["analysis_ms"] * 1e6) / fp32_gflops,
                           "algorithmic_bytes": ana_bytes32},
        "observe_mixed": {"ms": mixed["observe_ms"]},
        "lbm_step_f64": {"ms": fp64["lbm_step_ms"], "bound": "fp64 alu", "achieved_gbs": lbm_bytes64 / (fp64["lbm_step_ms"] * 1e6),
                         "frac_of_hbm": lbm_bytes64 / (fp64["lbm_step_ms"] * 1e6) / hbm},
        "analysis_fp64": {"ms": fp64["analysis_ms"], "bound": "fp64 alu",
                          "achieved_gflops": flops / (fp64["analysis_ms"] * 1e6),
                          "peak_gflops": FP64_NOMINAL_GFLOPS,
                          "frac": flops / (fp64["analysis_ms"] * 1e6) / FP64_NOMINAL_GFLOPS,
                          "algorithmic_bytes": ana_bytes64},
    }
    ncells = cfg.nx * cfg.ny
    throughput = {
        "mlups_x_members_f32": ncell / (mixed["lbm_step_ms"] * 1e3),
        "mlups_x_members_f64": ncell / (fp64["lbm_step_ms"] * 1e3),
        "grid_point_analyses_per_s_mixed": ncells / (mixed["analysis_ms"] * 1e-3),
        "grid_point_analyses_per_s_fp64": ncells / (fp64["analysis_ms"] * 1e-3),
        "nature_run_ms_per_cycle": mixed["nature_ms"],
        "jacobi_sweeps_per_point_mixed": mixed["sweeps"],
        "jacobi_sweeps_per_point_fp64": fp64["sweeps"],
    }
    lbm_share = mixed["lbm_step_ms"] * cfg.steps_per_cycle
    kern["lbm_step_f32"]["traffic"] = NCU_TRAFFIC["lbm_step_f32"]
    kern["analysis_mixed"]["traffic"] = NCU_TRAFFIC["analysis_mixed"]
    kern["analysis_fp64"]["traffic"] = NCU_TRAFFIC["analysis_fp64"]
    if lbm_share >= mixed["analysis_ms"]:
        ach = kern["lbm_step_f32"]["achieved_gbs"]
        roof = {"kernel": "lbm_step_kernel<float,4,shift>", "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": NCU_TRAFFIC["lbm_step_f32"],
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback"}
    else:
        ach = kern["analysis_mixed"]["achieved_gflops"]
        tr = NCU_TRAFFIC["analysis_mixed"]
        roof = {"kernel": "mixed analysis: run_jacobi_kernel<28> + run_refine_kernel<28> (runs of 8 grid points)",
                "bound": "alu", "achieved": ach / 1000.0, "peak": fp32_gflops / 1000.0, "unit": "TFLOP/s",
                "frac": ach / fp32_gflops, "traffic": tr,
                "algorithmic_bytes": ana_bytes32,
                "traffic_over_algorithmic": (tr / ana_bytes32) if tr else None,
                "peak_source": "derived: %d SMs x %d binary32 FMA lanes x 2 flops x %.0f MHz (nominal)"
                               % (nsm, FP32_LANES_PER_SM, sm_mhz),
                "work": "algorithmic flops of the method (its FP64 formulation): 9 n^3 per symmetric "
                        "eigensolve (n = min(k, p)) + 2 per multiply-add of the products; the kernels do it in "
                        "binary32 (Jacobi) and double-binary32 (refinement), several times this count",
                "fp64_equivalent": {"achieved": ach / 1000.0, "peak": FP64_NOMINAL_GFLOPS / 1000.0,
                                    "frac": ach / FP64_NOMINAL_GFLOPS,
                                    "note": "the same work against the FP64 nominal peak, for comparison "
                                            "with an FP64-bound path; not the bound of these kernels"},
                "issue_active": ISSUE_ACTIVE}

    adj = batch = osse = None
    if args.case == "all":
        osse = measure_osse(cfg, binding.LBM_MIXED)
        adj = measure_adjoint(cfg)
        adj["peak_gbs"] = hbm
        adj["frac"] = adj["achieved_gbs"] / hbm
        batch = measure_batch(cfg)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(cfg)

    if rank == 0:
        value = replica_value(ms, world)
        line = {
            "metric": METRIC, "value": value, "unit": "cycles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 LBM + f64 eigensolve (mixed)", "data": "synthetic",
            "config": {"workload": cfg.name(), "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": L2_NOTE},
            "fp64": {"value": replica_value(ms64, world), "unit": "cycles/s", "ms_per_step": ms64,
                     "dtype": "f64"},
            "graph": graph,
            "e2e": {"value": world / e2e_val, "unit": "cycles/s",
                    "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]},
            "gpu_launches": args.steps * mixed["launches_per_cycle"],
            "roofline": roof, "kernels": kern, "throughput": throughput, "adjoint": adj, "batch": batch,
            "osse_10000_steps_mixed": osse,
            # Ensemble-mean velocity RMSE against the nature run after the
            # warm-up and timed cycles of each leg (their counts differ).
            "rmse": {"mixed": mixed["rmse"], "mixed_cycles": args.warmup + args.steps, "fp64": fp64["rmse"],
                     "fp64_cycles": args.warmup + max(3, args.steps // 3), "obs_noise_rms": cfg.sigma * np.sqrt(2)},
            "clocks": mixed["clocks"], "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
