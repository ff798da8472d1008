"""The step loop as one CUDA graph launch (device-side Moulinec-Suquet loop
control through conditional nodes) and the batched form over instances with
different grids.  Both must reproduce the host-controlled path bitwise: the
kernels and their order are the same and every reduction has a fixed order."""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from parity_util import rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def workload(shape, vids, n_grains, seed, steps=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    R = I.shoemake_rotations(rng, n_grains) if n_grains > 1 else np.eye(3)[None]
    grain = I.voronoi_grains(rng, shape, n_grains) if n_grains > 1 else None
    f = I._place_nuclei(rng, shape, vids, grain, R, 3, semi_s=(2.0, 4.0), semi_tn=(1.0, 2.5))
    ep = I.gaussian_plastic_strain(rng, shape, 2.0, 0.002)
    d = rng.standard_normal(3)
    E = np.stack([I.uniaxial_strain(-0.006 * (k + 1) / steps, d) for k in range(steps)])
    return I.Workload(f"g{shape}", shape, list(vids), f, ep, grain, R, E)


def run(h, w, splits, inst=0, n_inst=1, Es=None):
    infos = []
    k = 0
    for n in splits:
        if n_inst == 1:
            code, info = h.step(w.E[k:k + n][None])
        else:
            code, info = h.step(np.stack([e[k:k + n] for e in Es]))
        infos.append((code, info))
        k += n
    return infos


@pytest.mark.parametrize("precision, tol", [("fp32", 1e-6), ("fp64", 1e-12), ("fp32", 0.0)])
def test_graph_mode_is_bitwise_equal_to_host_mode(precision, tol):
    w = workload((12, 16, 20), [0, 3], 2, seed=41)
    kw = dict(precision=precision, ms_tol=tol, ms_max_it=5 if tol == 0 else 100)
    he = pf.handle_for(w, **kw)
    hg = pf.handle_for(w, use_graph=1, **kw)
    # odd and even step counts across calls flip the f buffers between calls
    ie = run(he, w, [3, 2, 2])
    ig = run(hg, w, [3, 2, 2])
    for (ce, a), (cg, b) in zip(ie, ig):
        assert ce == cg == pf.PF_OK
        assert a[0].n_ms_last == b[0].n_ms_last and a[0].n_ms_total == b[0].n_ms_total
        assert a[0].resid == b[0].resid
        assert list(a[0].mean_sigma) == list(b[0].mean_sigma)
    fe, ee = he.get_fields(0)
    fg, eg = hg.get_fields(0)
    assert np.array_equal(fe, fg) and np.array_equal(ee, eg)
    me, se = he.stress(0)
    mg, sg = hg.stress(0)
    assert np.array_equal(se, sg) and np.array_equal(me, mg)
    assert np.array_equal(he.energy(0), hg.energy(0))
    he.close()
    hg.close()


def test_batch_of_uneven_grids_matches_single_runs_and_oracle():
    shapes = [(12, 16, 20), (10, 9, 15), (8, 8, 8)]
    ws = [workload(s, v, g, seed=50 + i, steps=4) for i, (s, v, g) in
          enumerate(zip(shapes, ([0], [1, 4], [2, 3, 5]), (2, 1, 3)))]
    hb = pf.batch_handle_for(ws, precision="fp64", ms_tol=1e-12, use_graph=1)
    code, infos = hb.step(np.stack([w.E for w in ws]))
    assert code == pf.PF_OK
    for i, w in enumerate(ws):
        hs = pf.handle_for(w, precision="fp64", ms_tol=1e-12)
        _, inf = hs.step(w.E[None])
        fb, eb = hb.get_fields(i)
        fs, es = hs.get_fields(0)
        assert np.array_equal(fb, fs) and np.array_equal(eb, es)
        assert infos[i].n_ms_total == inf[0].n_ms_total
        o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
        for k in range(4):
            o.step(w.E[k])
        assert rel_max(fb, o.f.reshape(w.V, -1)) <= 1e-12
        assert rel_max(eb, o.eps_voigt().reshape(6, -1)) <= 1e-12
        hs.close()
    hb.close()


def test_graph_mode_error_codes():
    w = workload((8, 8, 8), [0], 2, seed=60, steps=3)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-14, ms_max_it=2, use_graph=1)
    code, info = h.step(w.E[None], allow=(pf.PF_ENOCONV,))
    assert code == pf.PF_ENOCONV and info[0].status == pf.PF_ENOCONV
    assert info[0].n_ms_last == 2 and info[0].n_ms_total == 6
    h.close()
    bad = w.eps_p.copy()
    bad[0, 1, 2, 3] = np.nan
    w2 = I.Workload("nan", w.shape, w.variant_ids, w.f, bad, w.grain, w.grain_R, w.E)
    h = pf.handle_for(w2, precision="fp32", ms_tol=1e-6, use_graph=1)
    code, info = h.step(w.E[None], allow=(pf.PF_ENAN,))
    assert code == pf.PF_ENAN and info[0].status == pf.PF_ENAN
    h.close()
