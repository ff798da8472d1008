"""The plastic strain handed over from host memory every step, as the
staggered CP-FE/PF scheme does (Table Algorithm_PF): the upload runs on the
handle's own stream and pf_step overlaps it with its first kernels (C0, the
extrapolated warm start), joining it before the first pass that reads the
field.  A new field each step, from pageable and from pinned host memory,
eager and graph stepping, against the oracle given the same fields: FP64
within 1e-12, FP32 within 1e-5."""
import numpy as np
import pytest

from paper_2302_13612_gb300 import pf
from parity_util import Pair
from test_gpu_parity import custom_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


@pytest.mark.parametrize("precision,use_graph,pinned", [("fp64", 0, False), ("fp64", 1, False), ("fp32", 0, True),
                                                        ("fp32", 1, True)])
def test_new_plastic_strain_every_step(precision, use_graph, pinned):
    import torch
    w = custom_workload((12, 16, 20), [0, 3], 2, seed=97, steps=5, eps_p=True, nuclei=3)
    rng = np.random.Generator(np.random.PCG64(98))
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=3, warm_degree=3, use_graph=use_graph)
    dt = np.float64 if precision == "fp64" else np.float32
    host = torch.empty((6, w.nvox), dtype=torch.float64 if precision == "fp64" else torch.float32)
    if pinned:
        host = host.pin_memory()
    buf = host.numpy()
    for k in range(5):
        ep = (w.eps_p.reshape(6, -1) * (1.0 + 0.3 * k) + 1e-4 * rng.standard_normal((6, w.nvox)))
        buf[...] = ep.astype(dt)
        p.h.set_plastic_strain(0, buf)
        p.o.eps_p = buf.astype(np.float64).reshape((6,) + w.shape)
        p.step(k)
    e = p.errors()
    p.close()
    if precision == "fp64":
        assert e["f_max"] <= 1e-12 and e["eps_max"] <= 1e-12 and e["sigma_max"] <= 1e-12, e
    else:
        assert e["f_l2"] <= 1e-5 and e["eps_l2"] <= 1e-5 and e["sigma_l2"] <= 1e-5, e
