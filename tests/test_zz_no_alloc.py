"""The allocation-free residual entry point, pf_ms_residual_static.

Some callers cannot call cudaMalloc -- a host code that carves all device
memory out of one pool at start-up, or a user subroutine running inside
another solver that must not allocate on the GPU.  For them the library
offers this one reduction with its scratch in a fixed device array.  The
test checks it against the residual that pf_step reports for the same two
strain fields, on two calls in a row (the shared scratch array keeps the
previous call's contents), and that it refuses sizes beyond its limit.
This file is named to be collected last."""
import math

import numpy as np
import pytest

from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision, tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_static_residual_matches_pf_step(precision, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.Generator(np.random.PCG64(31))
    shape = (16, 20, 24)
    R = I.shoemake_rotations(rng, 2)
    grain = I.voronoi_grains(rng, shape, 2)
    f = I._place_nuclei(rng, shape, [0, 3], grain, R, 3)
    ep = I.gaussian_plastic_strain(rng, shape, 2.0, 0.002)
    E = np.stack([I.uniaxial_strain(-0.003 * (k + 1), I.D_10M10) for k in range(3)])
    w = I.Workload("static", shape, [0, 3], f, ep, grain, R, E)
    N = w.nvox
    # one Moulinec-Suquet pass per step: the residual pf_step reports for
    # step k compares the strain after step k with the strain after step k-1
    h = pf.handle_for(w, precision=precision, ms_tol=0.0, ms_max_it=1)
    dt = torch.float32 if precision == "fp32" else torch.float64
    code = pf.PF_FP32 if precision == "fp32" else pf.PF_FP64
    prev = torch.empty((6, N), device="cuda", dtype=dt)
    cur = torch.empty((6, N), device="cuda", dtype=dt)
    h.step(E[0][None, None, :])
    h.get_fields(0, None, prev, mem=pf.PF_MEM_DEVICE)
    torch.cuda.synchronize()
    for k in (1, 2):  # two calls in a row
        _, info = h.step(E[k][None, None, :])
        h.get_fields(0, None, cur, mem=pf.PF_MEM_DEVICE)
        torch.cuda.synchronize()
        rc, out = pf.ms_residual_static(cur, prev, N, code, None)
        assert rc == pf.PF_OK
        r = math.sqrt(out[0] / out[1])
        assert abs(r - info[0].resid) <= tol * info[0].resid, (k, r, info[0].resid)
        prev.copy_(cur)
    rc, _ = pf.ms_residual_static(cur, prev, 67108864 + 1, code, None)
    assert rc == pf.PF_EINVAL
    h.close()
