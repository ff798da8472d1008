"""Checks at the full 256^3 polycrystal size with six variants, in the launch
configuration that bench.py times: properties that hold at any size, stress
recomputed by the oracle at sampled voxels, and FP32 against the FP64 GPU
step (which matches the oracle at the smaller sizes)."""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from parity_util import rel_l2, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = I.config3(steps=2)
    out = {"w": w}
    for prec, tol in (("fp32", 1e-6), ("fp64", 1e-10)):
        h = pf.handle_for(w, precision=prec, ms_tol=tol, ms_max_it=200)
        code, info = h.step(w.E[:1][None])
        assert code == pf.PF_OK
        f_n, _ = h.get_fields(0)
        code, info = h.step(w.E[1:2][None])
        assert code == pf.PF_OK
        f_next, eps = h.get_fields(0)
        mean, sig = h.stress(0)
        out[prec] = dict(f_n=f_n, f=f_next, eps=eps, sig=sig, mean=mean, info=info[0])
        h.close()
    return out


def test_mean_strain_is_prescribed(runs):
    w = runs["w"]
    for prec, tol in (("fp32", 1e-6), ("fp64", 1e-12)):
        eps = runs[prec]["eps"]
        assert np.abs(eps.astype(np.float64).mean(axis=1) - w.E[1]).max() <= tol * 0.02


def test_sampled_stress_matches_oracle_pointwise(runs):
    w = runs["w"]
    rng = np.random.default_rng(5)
    idx = rng.choice(w.nvox, size=4096, replace=False)
    tab = O.build_tables(w.C_hex, w.c_over_a, w.variant_ids, w.grain_R, w.twin_stiffness)
    for prec, tol in (("fp32", 2e-6), ("fp64", 1e-13)):
        r = runs[prec]
        f = r["f_n"][:, idx].astype(np.float64)[:, None, None, :]
        eps = O.voigt_to_tensor2(r["eps"][:, idx].astype(np.float64))[:, :, None, None, :]
        g = w.grain.reshape(-1)[idx][None, None, :]
        e = eps - O.eigenstrain(f, None, g, tab, w.gamma_tw)
        ref = O.tensor2_to_voigt(O.stress(f, e, g, tab)).reshape(6, -1)
        assert rel_max(r["sig"][:, idx], ref) <= tol


def test_stress_is_equilibrated(runs):
    torch = pytest.importorskip("torch")
    w = runs["w"]
    nz, ny, nx = w.shape
    for prec, tol in (("fp32", 2e-5), ("fp64", 1e-9)):
        sig = torch.from_numpy(runs[prec]["sig"].reshape(6, nz, ny, nx)).to("cuda", torch.float64)
        sh = torch.fft.rfftn(sig, dim=(1, 2, 3))
        kz = torch.fft.fftfreq(nz, device="cuda", dtype=torch.float64)[:, None, None]
        ky = torch.fft.fftfreq(ny, device="cuda", dtype=torch.float64)[None, :, None]
        kx = torch.fft.rfftfreq(nx, device="cuda", dtype=torch.float64)[None, None, :]
        # Nyquist modes carry no strain fluctuation in the scheme; skip them
        keep = (kz.abs() < 0.5) & (ky.abs() < 0.5) & (kx.abs() < 0.5)
        P = [(0, 5, 4), (5, 1, 3), (4, 3, 2)]
        worst = 0.0
        for i in range(3):
            div = sh[P[i][0]] * kx + sh[P[i][1]] * ky + sh[P[i][2]] * kz
            div = torch.where(keep, div, torch.zeros_like(div))
            worst = max(worst, float(div.abs().max()))
        scale = float(sh[:, 1:].abs().max()) * 0.5
        assert worst / scale <= tol, (prec, worst / scale)


def test_fp32_matches_fp64_gpu_step(runs):
    a, b = runs["fp32"], runs["fp64"]
    assert rel_l2(a["sig"], b["sig"]) <= 1e-5
    assert rel_l2(a["f"], b["f"]) <= 1e-5
    assert rel_max(a["mean"], b["mean"]) <= 1e-5
