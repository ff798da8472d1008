"""Pad layer (a low-mobility region around the sample, Sec. 3 and 4; the
oracle's reading R11) on the CUDA path against the FP64 oracle: corrections
on the reference mobility, FP64 within 1e-12, FP32 within 1e-5, unit
mobility equal to the plain step, a frozen zero-mobility pad, graph and
host-controlled loops bitwise equal, invalid fields refused."""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from parity_util import Pair, rel_l2, rel_max
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def padded(shape, seed, low=1e-3, width=2, steps=4, vids=(0, 3)):
    w = custom_workload(shape, list(vids), 1, seed=seed, steps=steps)
    w.mobility = I.pad_mobility(shape, (width, width, width), low)
    w.f = w.f * (w.mobility == 1.0)
    return w


@pytest.mark.parametrize("shape", [(20, 12, 16), (10, 9, 15)])
def test_fp64_fixed_passes(shape):
    w = padded(shape, seed=61)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=5, mob_corr=3)
    for k in range(4):
        code, info, oi = p.step(k)
        assert abs(info.mob_change - oi["mob_change"]) <= 1e-9 * oi["mob_change"] + 1e-300
    e = p.errors()
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve") and not v <= FP64_TOL}
    assert not bad, (bad, e)
    p.close()


def test_unit_mobility_is_the_plain_step():
    w = padded((12, 16, 20), seed=62, low=1.0)
    a = Pair(w, "fp64", ms_tol=0.0, ms_max_it=4, mob_corr=2)
    w2 = padded((12, 16, 20), seed=62, low=1.0)
    w2.mobility = None
    b = Pair(w2, "fp64", ms_tol=0.0, ms_max_it=4)
    a.run(3)
    b.run(3)
    fa, ea = a.h.get_fields(0)
    fb, eb = b.h.get_fields(0)
    assert rel_max(fa, fb) <= 1e-13 and rel_max(ea, eb) <= 1e-13
    a.close()
    b.close()


def test_zero_mobility_pad_is_frozen():
    w = padded((16, 12, 20), seed=63, low=0.0)
    N = w.nvox
    pad = (w.mobility == 0.0).reshape(N)
    h = pf.handle_for(w, precision="fp64", ms_tol=0.0, ms_max_it=4, mob_corr=30)
    f0, _ = h.get_fields(0)
    _, info = h.step(w.E[None, 0:3])
    f, _ = h.get_fields(0)
    assert np.abs(f[:, pad] - f0[:, pad]).max() <= 1e-10
    assert np.abs(f[:, ~pad] - f0[:, ~pad]).max() > 1e-4
    assert info[0].mob_change <= 1e-12
    h.close()


def test_fp32_pillar_with_pad():
    w = I.pillar_pad(steps=3)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-6, mob_corr=3)
    o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, n_corr=3)
    for k in range(3):
        code, info = h.step(w.E[k][None, None, :])
        assert code == pf.PF_OK
        oi = o.step(w.E[k])
        assert rel_max(np.array(info[0].mean_sigma[:]), oi["mean_sigma"]) <= FP32_TOL
    f, _ = h.get_fields(0)
    assert rel_l2(f, o.f.reshape(w.V, -1)) <= FP32_TOL
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_equals_eager(precision):
    w = padded((16, 12, 20), seed=64)
    kw = dict(precision=precision, ms_tol=1e-9 if precision == "fp64" else 1e-5, ms_max_it=60, mob_corr=2)
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    _, ie = he.step(w.E[None, 0:4])
    _, ig = hg.step(w.E[None, 0:4])
    assert ie[0].mob_change == ig[0].mob_change
    for x, y in zip(he.get_fields(0), hg.get_fields(0)):
        assert np.array_equal(x, y)
    he.close()
    hg.close()


def test_invalid_mobility_refused():
    w = padded((8, 8, 8), seed=65)
    h = pf.handle_for(w, precision="fp32")
    bad = np.ones(w.nvox, dtype=np.float32)
    bad[3] = 1.5
    assert h.lib.pf_set_mobility(h.h, 0, bad.ctypes.data, pf.PF_MEM_HOST) == pf.PF_EINVAL
    bad[3] = np.nan
    assert h.lib.pf_set_mobility(h.h, 0, bad.ctypes.data, pf.PF_MEM_HOST) == pf.PF_EINVAL
    h.close()
