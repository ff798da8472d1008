"""Extrapolated warm start of the Moulinec-Suquet passes on the CUDA path
against the FP64 oracle (its reading R9): FP64 within 1e-12 with fixed and
with converged passes for degrees 1-5, FP32 within 1e-5, a given strain
counting as one held solution, graph and host-controlled loops bitwise
equal, and fewer passes than the plain warm start on a smooth run."""
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


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_fp64_fixed_passes(degree):
    w = custom_workload((20, 12, 16), [0, 3], 2, seed=41, steps=8)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=5, warm_degree=degree)
    p.run(8)
    e = p.errors()
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve") and not v <= FP64_TOL}
    assert not bad, (bad, e)
    p.close()


def test_fp64_converged_same_pass_counts():
    w = custom_workload((10, 9, 15), [1, 2, 5], 3, seed=42, steps=5)
    p = Pair(w, "fp64", ms_tol=1e-12, ms_max_it=300, warm_degree=3)
    p.run(5)
    assert p.n_ms_gpu == p.n_ms_ora
    e = p.errors()
    assert e["eps_max"] <= FP64_TOL and e["f_max"] <= FP64_TOL and e["sigma_max"] <= FP64_TOL, e
    p.close()


def test_fp32_converged_pillar_recipe():
    w = I.config2(steps=8, n=32, total_steps=20)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-6, warm_degree=3)
    o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm_degree=3)
    for k in range(8):
        code, info = h.step(w.E[k][None, None, :])
        assert code == pf.PF_OK and info[0].resid <= 1e-6
        oi = o.step(w.E[k])
        assert rel_max(np.array(info[0].mean_sigma[:]), oi["mean_sigma"]) <= FP32_TOL
    mean, sig = h.stress(0)
    f, eps = h.get_fields(0)
    assert rel_l2(sig, O.tensor2_to_voigt(o.stress_field()).reshape(6, -1)) <= FP32_TOL
    assert rel_l2(f, o.f.reshape(2, -1)) <= FP32_TOL
    h.close()


def test_given_strain_and_reset():
    w = custom_workload((12, 16, 20), [0, 3], 2, seed=43, steps=4)
    N = w.nvox
    kw = dict(precision="fp64", ms_tol=0.0, ms_max_it=4, warm_degree=2)
    a = pf.handle_for(w, **kw)
    a.step(w.E[None, 0:2])
    f1, e1 = a.get_fields(0)
    # restart from (f1, e1): the given strain is one held solution, as in the oracle
    a.set_fields(0, f1, w.eps_p.reshape(6, N), w.grain.reshape(N), e1)
    a.step(w.E[None, 2:4])
    o = O.State(f1.reshape((w.V,) + w.shape), w.eps_p, w.grain,
                O.build_tables(w.C_hex, w.c_over_a, w.variant_ids, w.grain_R, w.twin_stiffness, 0.0),
                O.Params(w.c1, w.c2, w.c3, w.dt, w.gamma_tw, 0.0, 4, True), e1.reshape((6,) + w.shape),
                None, 2)
    o.step(w.E[2])
    o.step(w.E[3])
    f, eps = a.get_fields(0)
    assert rel_max(eps, o.eps_voigt().reshape(6, N)) <= FP64_TOL
    assert rel_max(f, o.f.reshape(w.V, N)) <= FP64_TOL
    a.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_equals_eager(precision):
    w = custom_workload((16, 12, 20), [0, 3], 2, seed=44, steps=6)
    kw = dict(precision=precision, ms_tol=1e-9 if precision == "fp64" else 1e-5, ms_max_it=60, warm_degree=3)
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    _, ie = he.step(w.E[None, 0:6])
    _, ig1 = hg.step(w.E[None, 0:3])
    _, ig2 = hg.step(w.E[None, 3:6])
    assert ie[0].n_ms_total == ig1[0].n_ms_total + ig2[0].n_ms_total
    for x, y in zip(he.get_fields(0), hg.get_fields(0)):
        assert np.array_equal(x, y)
    he.close()
    hg.close()


def test_fewer_passes_on_a_smooth_run():
    w = I.config3(steps=10, n=32, seed=1003, n_grains=8)
    tot = {}
    for d in (0, 3):
        h = pf.handle_for(w, precision="fp32", ms_tol=1e-6, warm_degree=d)
        _, info = h.step(w.E[None, :])
        tot[d] = info[0].n_ms_total
        h.close()
    assert tot[3] < tot[0], tot


# ---- least-squares form (warm_points > warm_degree + 1) ----------------------
@pytest.mark.parametrize("degree,points", [(1, 4), (2, 5), (3, 6)])
def test_fp64_least_squares_fixed_passes(degree, points):
    w = custom_workload((20, 12, 16), [0, 3], 2, seed=45, steps=9)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=5, warm_degree=degree, warm_points=points)
    p.run(9)
    e = p.errors()
    bad = {k: v for k, v in e.items() if k in ("f_max", "eps_max", "sigma_max", "curve") and not v <= FP64_TOL}
    assert not bad, (bad, e)
    p.close()


def test_fp32_least_squares_pillar_recipe():
    w = I.config2(steps=10, n=32, total_steps=20)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-6, warm_degree=3, warm_points=6)
    o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm_degree=3, warm_points=6)
    for k in range(10):
        code, info = h.step(w.E[k][None, None, :])
        assert code == pf.PF_OK and info[0].resid <= 1e-6
        oi = o.step(w.E[k])
        assert rel_max(np.array(info[0].mean_sigma[:]), oi["mean_sigma"]) <= FP32_TOL
    f, eps = h.get_fields(0)
    assert rel_l2(f, o.f.reshape(2, -1)) <= FP32_TOL
    assert rel_l2(eps, o.eps_voigt().reshape(6, -1)) <= FP32_TOL
    h.close()


def test_least_squares_graph_equals_eager():
    w = custom_workload((16, 12, 20), [0, 3], 2, seed=46, steps=8)
    kw = dict(precision="fp32", ms_tol=1e-5, ms_max_it=60, warm_degree=2, warm_points=5)
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    _, ie = he.step(w.E[None, 0:8])
    _, ig1 = hg.step(w.E[None, 0:5])
    _, ig2 = hg.step(w.E[None, 5:8])
    assert ie[0].n_ms_total == ig1[0].n_ms_total + ig2[0].n_ms_total
    for x, y in zip(he.get_fields(0), hg.get_fields(0)):
        assert np.array_equal(x, y)
    he.close()
    hg.close()
