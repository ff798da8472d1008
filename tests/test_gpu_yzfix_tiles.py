"""The FP32 y and z passes with compile-time transform plans at every plan and
tile width they are built for: 256 = 16 x 16, 128 = 16 x 8 and 8 x 16,
64 = 8 x 8, the lengths with factors 3 and 5 of the batched workload,
80 = 16 x 5, 96 = 16 x 6, 120 = 12 x 10 and 160 = 16 x 10 (radices 6, 10
and 12 as prime-factor DFTs), and 512 = 16 x 32 (radix 32 as 2 x 16); y tiles of 8 and 16 columns, z tiles of 4 and
8 columns where a warp covers whole row groups of one component (the Green
operator of the Moulinec-Suquet solve and the Helmholtz solve of the update,
Eq. fRate3, both run in the z pass).  Between the two Stockham stages the
tile rows are swizzled within each 128-byte bank line; every combination is
checked against the FP64 oracle (relative L2 error <= 1e-5) on slabs whose
long axis is the transformed one, 24 voxels along x (13 half-spectrum
columns: two, four or one tile with a ragged tail).  The oracle runs once
per slab.  The x passes with compile-time plans of 80, 96, 120, 160 and 512
points (16 x 5, 16 x 6, 12 x 10 on 16 lanes, 16 x 10, 16 x 32, warp-local) on
slabs long along x.  The default plans (no radices forced) of 96, 120, 160
and 512 points are these in FP32; in FP64, and with the compile-time x
passes off, such a plan is refused."""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import pf
from parity_util import rel_l2
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu

PLANS = {256: ["16,16"], 128: ["16,8", "8,16"], 64: ["8,8"], 80: ["16,5"], 96: ["16,6"], 120: ["12,10"],
         160: ["16,10"], 512: ["16,32"]}


def built(n, radices, tw):
    # threads per pencil (n / smallest radix) times the tile width: whole warps
    return (n // min(int(r) for r in radices.split(",")) * tw) % 32 == 0


CASES = [(axis, n, r, tw) for axis, tws in (("y", (8, 16)), ("z", (4, 8))) for n in PLANS
         for r in PLANS[n] for tw in tws if built(n, r, tw) and (axis == "y" or n * 6 * tw * 8 <= 100 * 1024)]
# x: warp-local compile-time plans (the tile width does not apply)
CASES += [("x", n, r, 0) for n, r in ((80, "16,5"), (96, "16,6"), (120, "12,10"), (160, "16,10"), (256, "16,16"),
                                      (512, "16,32"))]
STEPS = 2
_ORACLE = {}


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def slab(axis, n):
    shape = {"x": (4, 6, n), "y": (4, n, 24), "z": (n, 4, 24)}[axis]
    return custom_workload(shape, [0, 1, 2, 3, 4, 5], 2, seed=60 + n + (axis == "z"), steps=STEPS, nuclei=3)


def oracle(axis, n, w):
    key = (axis, n)
    if key not in _ORACLE:
        o = O.state_from_workload(w, ms_tol=0.0, ms_max_it=3)
        for k in range(STEPS):
            o.step(w.E[k])
        sig = O.tensor2_to_voigt(o.stress_field()).reshape(6, w.nvox)
        _ORACLE[key] = (o.f.reshape(w.V, w.nvox), o.eps_voigt().reshape(6, w.nvox), sig)
    return _ORACLE[key]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}_r{c[2].replace(',', '-')}_tw{c[3]}")
def test_fixed_plan_tile(case, monkeypatch):
    axis, n, radices, tw = case
    w = slab(axis, n)
    monkeypatch.setenv("PF_RADIX_" + axis.upper(), radices)
    if axis != "x":
        monkeypatch.setenv("PF_Y_TX" if axis == "y" else "PF_Z_TZ", str(tw))
    h = pf.handle_for(w, precision="fp32", ms_tol=0.0, ms_max_it=3, autotune=0)
    try:
        for k in range(STEPS):
            h.step(w.E[k][None, None, :])  # raises on any error but the capped pass count
        f, eps = h.get_fields(0)
        _mean, sig = h.stress(0)
    finally:
        h.close()
    fo, eo, so = oracle(axis, n, w)
    e = {"f": rel_l2(f, fo), "eps": rel_l2(eps, eo), "sigma": rel_l2(sig, so)}
    assert all(v <= 1e-5 for v in e.values()), e


@pytest.mark.parametrize("axis,n", [(a, n) for a in "xyz" for n in (96, 120, 160, 512)])
def test_default_compile_time_plan(axis, n):
    """No radices forced: the FP32 axis of 96, 120, 160 or 512 points runs its
    compile-time plan; against the same oracle slab as the forced runs."""
    w = slab(axis, n)
    h = pf.handle_for(w, precision="fp32", ms_tol=0.0, ms_max_it=3, autotune=0)
    try:
        for k in range(STEPS):
            h.step(w.E[k][None, None, :])
        f, eps = h.get_fields(0)
        _mean, sig = h.stress(0)
    finally:
        h.close()
    fo, eo, so = oracle(axis, n, w)
    e = {"f": rel_l2(f, fo), "eps": rel_l2(eps, eo), "sigma": rel_l2(sig, so)}
    assert all(v <= 1e-5 for v in e.values()), e


@pytest.mark.parametrize("precision,env,n", [("fp64", {"PF_RADIX_Y": "16,6"}, 96), ("fp64", {"PF_RADIX_X": "16,6"}, 96),
                                              ("fp32", {"PF_RADIX_X": "12,10", "PF_X_FIX": "0"}, 120)])
def test_compile_time_radix_refused(precision, env, n, monkeypatch):
    """A radix of the compile-time passes only (6, 10, 12, 32) is refused
    where no compile-time pass runs it: every FP64 axis, and the x axis with
    the compile-time x passes off."""
    shape = (4, 8, n) if "PF_RADIX_X" in env else (4, n, 24)
    w = custom_workload(shape, [0, 3], 1, seed=5, steps=1, nuclei=1)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    with pytest.raises(Exception):
        h = pf.handle_for(w, precision=precision, autotune=0)
        h.close()
