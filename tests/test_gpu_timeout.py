"""The give-up path of the bounded device waits, without a GPU fault: a handle
created with PF_WAIT_POLLS=0 gives every first wait on a bulk or TMA copy no
poll at all, so each pass records the load error and leaves after draining
its copies in flight (the drain wait keeps its normal limit).  pf_step must
return PF_ETIMEOUT, pf_destroy must succeed, and a handle created afterwards
on the same context must step normally."""
import numpy as np
import pytest

from paper_2302_13612_gb300 import pf
from parity_util import Pair, rel_max
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


@pytest.mark.parametrize("precision,use_graph,shape", [
    ("fp32", 0, (12, 10, 16)), ("fp64", 0, (12, 10, 16)), ("fp32", 1, (12, 10, 16)),
    # nx = 64, ny = 64: the compile-time-plan x and y passes; nz = 64: the
    # z passes (Helmholtz components split over CTAs)
    ("fp32", 0, (4, 64, 64)), ("fp32", 1, (4, 64, 64)), ("fp32", 0, (64, 8, 16)), ("fp32", 1, (64, 8, 16))])
def test_zero_polls_report_timeout(precision, use_graph, shape, monkeypatch):
    # nx = 16: the x passes stage their rows with cp.async.bulk; y and z use TMA
    w = custom_workload(shape, [0, 3], 2, seed=71, steps=2)
    monkeypatch.setenv("PF_WAIT_POLLS", "0")
    h = pf.handle_for(w, precision=precision, ms_tol=1e-6, use_graph=use_graph)
    monkeypatch.delenv("PF_WAIT_POLLS")
    code, _info = h.step(w.E[None, 0:1], allow=(pf.PF_ETIMEOUT, pf.PF_ENAN, pf.PF_ENOCONV))
    assert code == pf.PF_ETIMEOUT
    h.close()
    # the context is intact: a fresh handle steps and matches the oracle
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=3)
    p.run(2)
    e = p.errors()
    p.close()
    assert e["eps_max"] <= (1e-12 if precision == "fp64" else 1e-5), e
