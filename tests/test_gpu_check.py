"""The PF_CHECK build (libpf_check.so): every kernel verifies, before it
touches shared memory, that the layout it derives from its arguments fits
the launch's dynamic shared memory and that its tile lies inside the field,
and reports PF_ECHECK otherwise.  Parity cases that cover the fixed-plan and
the generic passes, FP64, FP32 and the mixed arm, uniaxial loading and the
autotuner run against that library in a child process: every launch must
pass its checks and the results must still match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import numpy as np
from paper_2302_13612_gb300 import pf
from parity_util import Pair
from test_gpu_parity import custom_workload
lib = pf.load_library()
assert lib._name.endswith("libpf_check.so"), lib._name
cases = [
    ((6, 8, 256), [0, 1, 2, 3, 4, 5], 3, False, "fp32", {}),
    ((8, 256, 6), [0, 3], 2, True, "fp32", {}),
    ((8, 256, 16), [0, 3], 2, True, "mixed", {}),
    ((20, 12, 16), [0, 3], 2, True, "fp64", {}),
    ((10, 9, 15), [1, 2, 5], 3, True, "fp32", {}),
    ((32, 24, 40), [0, 3], 2, True, "fp32", {"autotune": 1}),
    ((16, 16, 64), [0], 1, True, "fp32", {"load_dir": [0.3, 0.2, 1.0]}),
    # compile-time plans of 120, 160 and 512 points (prime-factor radices,
    # 12 threads on 16 lanes, radix 32 and the two-CTA z kernel)
    ((4, 6, 160), [0, 3], 2, True, "fp32", {}),
    ((4, 6, 120), [1, 4], 2, True, "fp32", {}),
    ((4, 120, 24), [0, 3], 2, True, "fp32", {}),
    ((160, 4, 24), [0, 1, 2, 3, 4, 5], 2, False, "fp32", {}),
    ((4, 4, 512), [0, 3], 1, True, "fp32", {}),
    ((512, 4, 8), [0, 3], 1, True, "fp32", {}),
]
for shape, vids, grains, ep, prec, kw in cases:
    w = custom_workload(shape, vids, grains, seed=71 + sum(shape), steps=2, eps_p=ep, nuclei=3)
    p = Pair(w, prec, ms_tol=0.0, ms_max_it=3, **kw)
    p.run(2)
    e = p.errors()
    p.h.energy(0)
    p.close()
    tol = 1e-12 if prec == "fp64" else 1e-5
    key = "eps_max" if prec == "fp64" else "eps_l2"
    assert e[key] <= tol, (shape, prec, e)
print("check build ok")
"""


def test_check_build_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, PF_CHECK_BUILD="1")
    code = CHILD % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "check build ok" in r.stdout
