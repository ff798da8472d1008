"""Oracle parity of the transform lengths the full-size workloads use: a
256-point transform along x, y and z in turn (the 256^3 polycrystal's
radix-16 pairs) and a 512-point one along x (the 512^3 pillar, whose x
passes transform block-wide because 512 / smallest radix exceeds one warp),
on thin slabs the FP64 oracle finishes in seconds.

Each slab runs twice: with the autotuner (as bench.py runs) and with the pass
shapes and radix orders forced through the PF_* overrides to the ones the
tuner keeps at 256^3 (x staging budget 96 KB, y tiles of 8 columns in CTAs of
128 threads, z tiles of 8 columns in CTAs of 256 threads, radix 16 x 16).
FP64: relative max error <= 1e-12; FP32: relative L2 error <= 1e-5."""
import numpy as np
import pytest

from paper_2302_13612_gb300 import pf
from parity_util import Pair
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu

FORCED = {"PF_X_SMEM_KB": "96", "PF_Y_TX": "8", "PF_Y_THREADS": "128", "PF_Z_TZ": "8", "PF_Z_THREADS": "256"}
AXIS_ENV = ("PF_RADIX_X", "PF_RADIX_Y", "PF_RADIX_Z")

# (nz, ny, nx), long axis (0 = x), variants, grains, plastic strain, forced
# radices of the long axis, also run with the autotuner
SLABS = [
    ((6, 8, 256), 0, [0, 1, 2, 3, 4, 5], 3, False, "16,16", True),
    ((8, 256, 6), 1, [0, 1, 2, 3, 4, 5], 3, False, "16,16", True),
    ((256, 6, 8), 2, [0, 1, 2, 3, 4, 5], 3, False, "16,16", True),
    ((4, 4, 512), 0, [0, 3], 1, True, "16,16,2", True),
    ((4, 4, 512), 0, [0, 3], 1, True, "8,8,8", False),
]
CASES = [(s, "forced") for s in SLABS] + [(s, "tuned") for s in SLABS if s[6]]


def case_id(c):
    s, mode = c
    return "x".join(map(str, s[0][::-1])) + ("_tuned" if mode == "tuned" else "_r" + s[5].replace(",", "-"))


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def run(slab, precision, mode, monkeypatch):
    shape, axis, vids, grains, ep, radices, _tuned = slab
    w = custom_workload(shape, vids, grains, seed=91 + sum(shape), steps=3, eps_p=ep, nuclei=3)
    if mode == "forced":
        for k, v in FORCED.items():
            monkeypatch.setenv(k, v)
        monkeypatch.setenv(AXIS_ENV[axis], radices)
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=3, autotune=1 if mode == "tuned" else 0)
    p.run(3)
    e = p.errors()
    p.close()
    return e


@pytest.mark.parametrize("case", CASES, ids=case_id)
def test_fp64_long_axis(case, monkeypatch):
    e = run(case[0], "fp64", case[1], monkeypatch)
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve") and not v <= 1e-12}
    assert not bad, e


@pytest.mark.parametrize("case", CASES, ids=case_id)
def test_fp32_long_axis(case, monkeypatch):
    e = run(case[0], "fp32", case[1], monkeypatch)
    bad = {k: v for k, v in e.items() if k in ("f_l2", "eps_l2", "sigma_l2") and not v <= 1e-5}
    assert not bad, e
