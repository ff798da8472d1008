"""Uniaxial loading (displacement control along one axis, the other mean
stresses free; the compression of Sec. 4) on the CUDA path against the FP64
oracle: FP64 within 1e-12, FP32 within 1e-5, the mean stress uniaxial along
the load axis once the passes converge, the lateral mean strain carried from
call to call and reset by pf_set_fields, graph and host-controlled loops
bitwise equal."""
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


def frame_stress(mean_sigma, d):
    Q = O.load_frame(d)
    return Q @ O.voigt_to_tensor2(np.asarray(mean_sigma)) @ Q.T


@pytest.mark.parametrize("d", [(0.3, -0.5, 0.8), (1.0, 0.0, 0.0), (0.0, 0.1, 1.0)])
def test_fp64_fixed_passes(d):
    # two grains, two variants, plastic strain; load axes on both branches of
    # the frame construction (|d_z| above and below 0.9)
    w = custom_workload((20, 12, 16), [0, 3], 2, seed=31)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=8, load_dir=d)
    p.run(4)
    e = p.errors()
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve", "strain_curve")
           and not v <= FP64_TOL}
    assert not bad, (bad, e)
    p.close()


def test_fp64_converged_is_uniaxial():
    w = custom_workload((10, 9, 15), [1, 2, 5], 3, seed=32, steps=3, strain=-0.01)
    d = np.array([0.2, 0.7, -0.4])
    p = Pair(w, "fp64", ms_tol=1e-12, ms_max_it=300, load_dir=d)
    for k in range(3):
        code, info, oi = p.step(k)
        assert code == pf.PF_OK
        assert info.n_ms_last == oi["n_ms"]
        s = frame_stress(info.mean_sigma[:], d)
        lateral = np.abs(s - np.diag([0.0, 0.0, s[2, 2]])).max()
        assert lateral <= 1e-9 * abs(s[2, 2]), s
        # the axial strain is the prescribed d.E.d
        u = d / np.linalg.norm(d)
        Et = O.voigt_to_tensor2(np.asarray(info.mean_strain[:]))
        assert abs(u @ Et @ u - u @ O.voigt_to_tensor2(w.E[k]) @ u) <= 1e-14
    e = p.errors()
    assert e["eps_max"] <= FP64_TOL and e["sigma_max"] <= FP64_TOL and e["strain_curve"] <= FP64_TOL, e
    p.close()


def test_fp32_fixed_passes():
    w = custom_workload((24, 20, 18), [0, 1, 2, 3, 4, 5], 6, seed=33)
    p = Pair(w, "fp32", ms_tol=0.0, ms_max_it=8, load_dir=(1.0, 1.0, 0.5))
    p.run(4)
    e = p.errors()
    assert e["sigma_l2"] <= FP32_TOL and e["f_l2"] <= FP32_TOL and e["curve"] <= FP32_TOL, e
    assert e["strain_curve"] <= FP32_TOL, e
    p.close()


def test_carry_over_and_reset():
    """Two calls of two steps equal one call of four; pf_set_fields drops the
    carried lateral strain so the handle restarts like a fresh one."""
    w = custom_workload((12, 16, 20), [0, 3], 2, seed=34)
    kw = dict(precision="fp64", ms_tol=0.0, ms_max_it=6, load_dir=(0.0, 1.0, 0.0))
    a = pf.handle_for(w, **kw)
    a.step(w.E[None, 0:4])
    fa, ea = a.get_fields(0)
    b = pf.handle_for(w, **kw)
    b.step(w.E[None, 0:2])
    b.step(w.E[None, 2:4])
    fb, eb = b.get_fields(0)
    assert np.array_equal(fa, fb) and np.array_equal(ea, eb)
    # restart a from the workload's fields: same as a fresh handle's first step
    N = w.nvox
    a.set_fields(0, w.f.reshape(w.V, N), w.eps_p.reshape(6, N), w.grain.reshape(N))
    _, ia = a.step(w.E[None, 0:1])
    c = pf.handle_for(w, **kw)
    _, ic = c.step(w.E[None, 0:1])
    assert np.array_equal(np.array(ia[0].mean_strain[:]), np.array(ic[0].mean_strain[:]))
    assert np.array_equal(a.get_fields(0)[1], c.get_fields(0)[1])
    for h in (a, b, c):
        h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_equals_eager(precision):
    w = custom_workload((16, 12, 20), [0, 3], 2, seed=35)
    kw = dict(precision=precision, ms_tol=1e-9 if precision == "fp64" else 1e-5, ms_max_it=60,
              load_dir=(0.4, 0.1, 0.9))
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    _, ie = he.step(w.E[None, 0:4])
    _, ig1 = hg.step(w.E[None, 0:2])
    _, ig2 = hg.step(w.E[None, 2:4])
    assert ie[0].n_ms_total == ig1[0].n_ms_total + ig2[0].n_ms_total
    assert np.array_equal(np.array(ie[0].mean_strain[:]), np.array(ig2[0].mean_strain[:]))
    for x, y in zip(he.get_fields(0), hg.get_fields(0)):
        assert np.array_equal(x, y)
    he.close()
    hg.close()
