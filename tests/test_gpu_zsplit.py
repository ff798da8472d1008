"""The per-component z passes (Helmholtz solve of the update, Eq. fRate3)
with the components split over CTAs in PF_Z_SPLIT groups (1: none):
the compile-time z plans (64-, 128- and 256-point z axes), isotropic and
anisotropic gradient coefficients (Table 5; per-component tensors offset by
the CTA's first component), three and six variants; each component's
arithmetic is unchanged, so the split runs match the unsplit ones bit for
bit and the oracle within the FP32 bound."""
import numpy as np
import pytest

from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from parity_util import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def crystal(shape, vids, seed, steps=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    R = I.shoemake_rotations(rng, 1)
    f = I._place_nuclei(rng, shape, vids, None, R, 4, semi_s=(2.0, 4.0), semi_tn=(1.0, 2.5))
    d = rng.standard_normal(3)
    E = np.stack([I.uniaxial_strain(-0.006 * (k + 1) / steps, d) for k in range(steps)])
    return I.Workload(f"crystal{shape}", shape, list(vids), f, None, None, R, E)


def run(w, split, aniso, monkeypatch):
    monkeypatch.setenv("PF_Z_SPLIT", str(split))
    c2 = (w.c2, 10 * w.c2, 10 * w.c2) if aniso else None
    p = Pair(w, "fp32", ms_tol=0.0, ms_max_it=3, c2_nst=c2)
    p.run(3)
    e = p.errors()
    f, eps, _fo, _eo = p.fields()
    p.close()
    return e, f, eps


# (nz, ny, nx)
@pytest.mark.parametrize("shape,vids", [((256, 4, 8), [0, 1, 2, 3, 4, 5]), ((128, 6, 8), [0, 2, 4]),
                                        ((64, 8, 6), [1, 3, 5])])
@pytest.mark.parametrize("aniso", [False, True])
def test_split_matches_unsplit_and_oracle(shape, vids, aniso, monkeypatch):
    w = crystal(shape, vids, seed=91 + shape[0])
    _e0, f0, eps0 = run(w, 1, aniso, monkeypatch)
    for split in (2, 3):
        e, f, eps = run(w, split, aniso, monkeypatch)
        assert np.array_equal(f, f0) and np.array_equal(eps, eps0), split
        assert e["f_l2"] <= 1e-5 and e["eps_l2"] <= 1e-5 and e["sigma_l2"] <= 1e-5, (split, e)

