"""Autotuned pass shapes and FFT radix orders: the tuned solver still
matches the FP64 oracle (other tiles and plans than the built-in ones), the
FP32 tuned step agrees with the built-in one, and the tuning file written by
one process is read by the next."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2302_13612_gb300 import pf
from parity_util import Pair, rel_l2
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


@pytest.mark.parametrize("shape", [(20, 12, 16), (32, 24, 40)])
def test_fp64_parity_after_tuning(shape):
    w = custom_workload(shape, [0, 3], 2, seed=81)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=5)
    p.h.close()
    p.h = pf.handle_for(w, precision="fp64", ms_tol=0.0, ms_max_it=5, autotune=1)
    p.run(3)
    e = p.errors()
    assert e["f_max"] <= 1e-12 and e["eps_max"] <= 1e-12 and e["sigma_max"] <= 1e-12, e
    p.close()


def test_fp32_tuned_matches_built_in():
    w = custom_workload((64, 48, 40), [0, 1, 2], 3, seed=82)
    a = pf.handle_for(w, precision="fp32", ms_tol=1e-6)
    b = pf.handle_for(w, precision="fp32", ms_tol=1e-6, autotune=1)
    a.step(w.E[None, 0:3])
    b.step(w.E[None, 0:3])
    fa, ea = a.get_fields(0)
    fb, eb = b.get_fields(0)
    assert rel_l2(fb, fa) <= 1e-5 and rel_l2(eb, ea) <= 1e-5
    a.close()
    b.close()


def test_tune_file_round_trip(tmp_path):
    path = tmp_path / "tune.txt"
    code = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from paper_2302_13612_gb300 import pf\n"
        "from test_gpu_parity import custom_workload\n"
        "w = custom_workload((16, 12, 20), [0], 1, seed=83)\n"
        "h = pf.handle_for(w, precision='fp32', autotune=1)\n"
        "h.step(w.E[None, 0:1])\n"
        "h.close()\n" % (ROOT, os.path.join(ROOT, "tests")))
    env = dict(os.environ, PF_TUNE_FILE=str(path))
    for _ in range(2):
        subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=300)
    lines = [l for l in path.read_text().splitlines() if l.strip()]
    assert len(lines) == 1, lines  # the second process found the shapes in the file
    v = [int(t) for t in lines[0].split()]
    assert v[:7] == [20, 12, 16, 1, 1, 1, 0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_cta_passes_parity(monkeypatch, precision):
    # the y and z passes in CTAs of 128 threads (an autotuner candidate),
    # with y tiles wider than one round of those threads
    monkeypatch.setenv("PF_Y_THREADS", "128")
    monkeypatch.setenv("PF_Z_THREADS", "128")
    monkeypatch.setenv("PF_Y_TX", "16")
    w = custom_workload((32, 24, 40), [0, 3], 2, seed=84)
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=4)
    p.run(3)
    e = p.errors()
    if precision == "fp64":
        assert e["f_max"] <= 1e-12 and e["eps_max"] <= 1e-12 and e["sigma_max"] <= 1e-12, e
    else:
        assert e["f_l2"] <= 1e-5 and e["eps_l2"] <= 1e-5 and e["sigma_l2"] <= 1e-5, e
    p.close()
