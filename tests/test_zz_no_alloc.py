"""The allocation-free analysis entry point gives the context path's result.

letkf_analyze_noalloc serves callers that cannot allocate device memory
(their memory manager owns the device pool, or an allocation's implicit
synchronisation is not allowed where they call from). It keeps its
intermediates in a fixed device array instead of context buffers. Here it
runs on a caller-owned CUDA tensor, through the C ABI, two calls in a row,
and each result is compared with letkf_observe + letkf_analyze on a context
holding the same ensemble, and the first also with the FP64 oracle. This
file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2308_03972_gb300 import inputs
from _helpers import TOL_FP64, U_RMS, norm_rel, osse_observations, turbulent_state

pytestmark = pytest.mark.gpu
TAU0, CS, MU = 0.55, 0.2, 6.16e-7
SIGMA = 0.1 * U_RMS


@pytest.mark.parametrize("nx,ny,k,nobs,d_cut", [(48, 40, 32, 4, 8.0), (32, 32, 8, 4, 8.0)])
def test_noalloc_analysis_matches_context_path_twice(gpu, nx, ny, k, nobs, d_cut):
    import torch

    f0 = turbulent_state(oracle, nx, ny, k, seed=k)
    force = inputs.forcing_field(nx, ny, seed=3, amp=3.5e-6)
    f0 = oracle.lbm_run(f0, force, TAU0, CS, MU, 3)
    obs = []
    for c in (1, 2):
        tu, tv = inputs.random_velocity(nx, ny, 100 + c, U_RMS)
        obs.append(osse_observations(nx, ny, nobs, nobs, 4, c, tu, tv, SIGMA))

    # Existing path: a context, letkf_observe + letkf_analyze, twice.
    refs = []
    with gpu.Ensemble(nx, ny, k, TAU0, CS, MU, gpu.LBM_FP64, f0=f0) as e:
        for ix, iy, yu, yv in obs:
            e.observe(ix, iy, yu, yv, SIGMA, SIGMA)
            e.analyze(d_cut, 1.05)
            refs.append(e.get_f())
        e.sync()

    # New path: the caller owns the state; no context, no allocation inside.
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    for (ix, iy, yu, yv), ref in zip(obs, refs):
        gpu.letkf_analyze_noalloc(f, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)
        torch.cuda.synchronize()
        assert norm_rel(f.cpu().numpy(), ref) <= TOL_FP64
    assert norm_rel(refs[1], refs[0]) > 1e-9  # the second call did new work
    ix, iy, yu, yv = obs[0]
    assert norm_rel(refs[0], oracle.letkf_analyze(f0, ix, iy, yu, yv, SIGMA, SIGMA, d_cut, 1.05)) <= TOL_FP64


def test_noalloc_rejects_sizes_beyond_its_limits(gpu):
    import torch

    f = torch.zeros((9, 4, 4, 2), dtype=torch.float64, device="cuda")
    n = 257
    ix = np.zeros(n, np.int32)
    with pytest.raises(gpu.LbmError) as err:
        gpu.letkf_analyze_noalloc(f, ix, ix, np.zeros(n), np.zeros(n), 0.1, 0.1, 2.0, 1.0)
    assert err.value.code == gpu.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_POINTS" in gpu.lbm_last_error(None)
    f = torch.zeros((9, 4, 4, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.LbmError) as err:
        gpu.letkf_analyze_noalloc(f, ix[:1], ix[:1], [0.0], [0.0], 0.1, 0.1, 2.0, 1.0)
    assert err.value.code == gpu.LBM_EINVAL


def test_noalloc_refuses_local_problems_above_64(gpu):
    """More than 64 members with dense observations: min(k, 2p) > 64 at
    some grid point, which the FP64 analysis does not hold."""
    import torch

    nx = ny = 32
    k = 128
    f0 = turbulent_state(oracle, nx, ny, k, seed=3)
    tu, tv = inputs.random_velocity(nx, ny, 5, U_RMS)
    ix, iy, yu, yv = osse_observations(nx, ny, 8, 8, 4, 1, tu, tv, SIGMA)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.LbmError) as err:
        gpu.letkf_analyze_noalloc(f, ix, iy, yu, yv, SIGMA, SIGMA, 8.0, 1.05)
    assert err.value.code == gpu.LBM_EINVAL
    with pytest.raises(ValueError):
        gpu.letkf_analyze_noalloc(f, ix, iy[:-1], yu, yv, SIGMA, SIGMA, 8.0, 1.05)
