"""The CUDA path (through the C ABI) on a two-phase laminate against the
closed forms of tests/laminate.py, with no oracle in between: one
Moulinec-Suquet pass from eps = E (which depends on the mixture stiffness of
Eq. stiffM, the twin eigenstrain, the reference medium C0 = <C(x)> and the
Green operator) and the converged solve (the exact laminate: continuous
traction and in-plane strain).  Layers normal to x, y and z on odd grids."""
import numpy as np
import pytest

import laminate as L
from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from test_oracle_laminate import laminate_case, layer_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def workload(c):
    return I.Workload("laminate", c["shape"], c["vids"], c["f"], c["ep"], c["grain"], c["Rs"], c["E"][None])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_first_pass_closed_form(axis, precision, tol):
    c = laminate_case(axis)
    h = pf.handle_for(workload(c), precision=precision, ms_tol=0.0, ms_max_it=1)
    h.step(c["E"][None, None])
    _f, eps = h.get_fields(0, want_f=False)
    h.close()
    C0 = sum(p * C for (p, C, _s) in c["layers"])
    eA, eB = L.first_pass(c["layers"], c["E"], axis, C0)
    expect = layer_field(c, eA, eB).reshape(6, -1)
    err = np.abs(eps.astype(np.float64) - expect).max() / np.abs(expect).max()
    assert err <= tol, err


@pytest.mark.parametrize("precision,tol,ms_tol", [("fp64", 1e-12, 1e-15), ("fp32", 1e-5, 1e-6)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_converged_closed_form(axis, precision, tol, ms_tol):
    c = laminate_case(axis)
    h = pf.handle_for(workload(c), precision=precision, ms_tol=ms_tol, ms_max_it=400)
    code, info = h.step(c["E"][None, None])
    assert code == pf.PF_OK and info[0].n_ms_last < 400
    _f, eps = h.get_fields(0, want_f=False)
    mean, sig = h.stress(0)
    h.close()
    eA, eB = L.converged(c["layers"], c["E"], axis)
    expect = layer_field(c, eA, eB).reshape(6, -1)
    err = np.abs(eps.astype(np.float64) - expect).max() / np.abs(expect).max()
    assert err <= tol, err
    # the traction sigma . n is uniform across the layers
    idx = L.TRACTION[axis]
    t = sig.astype(np.float64)[idx]
    spread = np.abs(t - t.mean(axis=1, keepdims=True)).max() / np.abs(sig).max()
    assert spread <= 10 * tol, spread
