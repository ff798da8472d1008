"""The mixed-precision arm (PF_MIXED): FP32 fields with the radix-16 stages of
the y transforms on the BF16 tensor cores (FP32 operands split exactly into
BF16 terms, FP32 accumulation).  Against the FP64 oracle on grids whose y
axis is 256 points long (the plan the tensor-core pass implements): relative
L2 error <= 1e-5 on f, the strain and the stress, as for FP32; and the pass
really runs on the tensor cores: the two-term split (PF_TC_TERMS=2, products
hh, hm, mh) changes the result, and its error is larger."""
import numpy as np
import pytest

from paper_2302_13612_gb300 import pf
from parity_util import Pair, rel_l2
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def run(shape, vids, grains, ep, precision, terms, monkeypatch, tuned=0):
    if terms is not None:
        monkeypatch.setenv("PF_TC_TERMS", str(terms))
    w = custom_workload(shape, vids, grains, seed=61 + sum(shape), steps=3, eps_p=ep, nuclei=3)
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=3, autotune=tuned)
    p.run(3)
    e = p.errors()
    f, eps, _fo, _eo = p.fields()
    p.close()
    return e, f, eps


@pytest.mark.parametrize("shape,vids,grains,ep", [
    ((8, 256, 6), [0, 1, 2, 3, 4, 5], 3, False),
    ((4, 256, 16), [0, 3], 1, True),
])
def test_mixed_matches_oracle(shape, vids, grains, ep, monkeypatch):
    e, f3, eps3 = run(shape, vids, grains, ep, "mixed", 3, monkeypatch)
    assert e["f_l2"] <= 1e-5 and e["eps_l2"] <= 1e-5 and e["sigma_l2"] <= 1e-5, e
    e2, f2, eps2 = run(shape, vids, grains, ep, "mixed", 2, monkeypatch)
    assert not np.array_equal(eps2, eps3)
    assert e2["eps_l2"] > e["eps_l2"], (e2, e)


def test_mixed_tuned(monkeypatch):
    e, _f, _eps = run((8, 256, 6), [0, 1, 2, 3, 4, 5], 3, False, "mixed", None, monkeypatch, tuned=1)
    assert e["f_l2"] <= 1e-5 and e["eps_l2"] <= 1e-5 and e["sigma_l2"] <= 1e-5, e
