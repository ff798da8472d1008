"""The iterated phase-field update (Eq. fRate3/4's i-loop with the
conservation loop's projection; the oracle's reading R12) on the CUDA path
against the FP64 oracle: FP64 within 1e-12 (alone, with the projection, with
the pad layer), FP32 within 1e-5, graph and host-controlled loops bitwise
equal."""
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


def check64(p):
    e = p.errors()
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve") and not v <= FP64_TOL}
    assert not bad, (bad, e)


@pytest.mark.parametrize("clamp", [0, 1])
def test_fp64_fixed_passes(clamp):
    w = custom_workload((20, 12, 16), [0, 3], 2, seed=71)
    w.dt = 0.8  # a long step: the i-loop matters and f leaves [0, 1] without the projection
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=5, pic_iters=4, clamp=clamp)
    for k in range(4):
        code, info, oi = p.step(k)
        assert abs(info.pic_change - oi["pic_change"]) <= 1e-9 * oi["pic_change"]
    check64(p)
    f, _ = p.h.get_fields(0)
    if clamp:
        assert f.min() >= 0.0 and f.max() <= 1.0 and f.sum(axis=0).max() <= 1.0 + 1e-15
    p.close()


def test_fp64_with_pad_layer():
    w = custom_workload((10, 9, 15), [1, 2], 1, seed=72)
    w.mobility = I.pad_mobility(w.shape, (2, 2, 2), 1e-3)
    w.f = w.f * (w.mobility == 1.0)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=4, pic_iters=3, mob_corr=2)
    p.run(3)
    check64(p)
    p.close()


def test_fp32_converged():
    w = custom_workload((24, 20, 18), [0, 1, 2, 3, 4, 5], 6, seed=73, steps=4)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-6, pic_iters=3)
    o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, n_pic=3)
    for k in range(4):
        code, info = h.step(w.E[k][None, None, :])
        assert code == pf.PF_OK
        oi = o.step(w.E[k])
        assert rel_max(np.array(info[0].mean_sigma[:]), oi["mean_sigma"]) <= FP32_TOL
    f, _ = h.get_fields(0)
    assert rel_l2(f, o.f.reshape(w.V, -1)) <= FP32_TOL
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_equals_eager(precision):
    w = custom_workload((16, 12, 20), [0, 3], 2, seed=74)
    kw = dict(precision=precision, ms_tol=1e-9 if precision == "fp64" else 1e-5, ms_max_it=60, pic_iters=3,
              clamp=1)
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    _, ie = he.step(w.E[None, 0:4])
    _, ig = hg.step(w.E[None, 0:4])
    assert ie[0].pic_change == ig[0].pic_change
    for x, y in zip(he.get_fields(0), hg.get_fields(0)):
        assert np.array_equal(x, y)
    he.close()
    hg.close()
