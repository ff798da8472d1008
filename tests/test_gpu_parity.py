"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64: relative error <= 1e-12 (max norm over the field); FP32: relative L2
error <= 1e-5 on stress and order parameter, as the target of the build
states.  Sizes span several tiles of every pass and leave ragged tails
(half-spectrum rows of odd length, row counts not divisible by the rows per
CTA, mixed radices 2/3/4/5/8/16, odd and even grids)."""
import math

import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I
from paper_2302_13612_gb300 import pf
from parity_util import Pair, rel_l2, rel_max

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pf.load_library()


def custom_workload(shape, vids, n_grains, seed, steps=4, eps_p=True, nuclei=4, strain=-0.006):
    rng = np.random.Generator(np.random.PCG64(seed))
    R = I.shoemake_rotations(rng, n_grains) if n_grains > 1 else np.eye(3)[None]
    grain = I.voronoi_grains(rng, shape, n_grains) if n_grains > 1 else None
    f = I._place_nuclei(rng, shape, vids, grain, R, nuclei, semi_s=(2.0, 4.0), semi_tn=(1.0, 2.5))
    ep = I.gaussian_plastic_strain(rng, shape, 2.0, 0.002) if eps_p else None
    d = rng.standard_normal(3)
    E = np.stack([I.uniaxial_strain(strain * (k + 1) / steps, d) for k in range(steps)])
    return I.Workload(f"custom{shape}", shape, list(vids), f, ep, grain, R, E)


def check(e, tol, keys=("f_max", "eps_max", "sigma_max", "curve")):
    bad = {k: v for k, v in e.items() if k in keys and not v <= tol}
    assert not bad, (bad, e)


def test_fp64_config1_full_run():
    """The plain-method workload: 32^3, one variant, homogeneous stiffness,
    -0.5% along [10-10], 100 steps, FP64."""
    w = I.config1()
    p = Pair(w, "fp64")
    p.run(100)
    e = p.errors()
    check(e, FP64_TOL)
    assert p.n_ms_gpu == p.n_ms_ora
    g = p.h.energy(0)
    go = np.array(p.o.energy())
    assert rel_max(g, go) <= FP64_TOL, (g, go)
    p.close()


def test_fp64_heterogeneous_mixed_radix_fixed_passes():
    # nx = 16 (radix 16), ny = 12 (4 x 3), nz = 20 (4 x 5); two grains, two
    # variants with rotated twin stiffness, plastic strain; 8 fixed passes.
    w = custom_workload((20, 12, 16), [0, 3], 2, seed=11)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=8)
    p.run(4)
    check(p.errors(), FP64_TOL)
    p.close()


def test_fp64_odd_grid_three_variants_converged():
    # nx = 15 (5 x 3, odd: no Nyquist column), ny = 9 (3 x 3), nz = 10 (2 x 5)
    w = custom_workload((10, 9, 15), [1, 2, 5], 3, seed=12, steps=3)
    p = Pair(w, "fp64", ms_tol=1e-13, ms_max_it=200)
    p.run(3)
    check(p.errors(), FP64_TOL)
    assert p.n_ms_gpu == p.n_ms_ora
    p.close()


def test_fp64_polycrystal_six_variants():
    w = custom_workload((24, 24, 24), [0, 1, 2, 3, 4, 5], 6, seed=13, steps=3, eps_p=False, nuclei=6)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=6)
    p.run(3)
    check(p.errors(), FP64_TOL)
    g = p.h.energy(0)
    assert rel_max(g, np.array(p.o.energy())) <= FP64_TOL
    p.close()


def test_fp64_large_radix_rows_ragged():
    # nx = 96 (8 x 4 x 3), ny = 5, nz = 3: 15 rows, not a multiple of the rows per CTA
    w = custom_workload((3, 5, 96), [4], 1, seed=14, steps=2)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=4)
    p.run(2)
    check(p.errors(), FP64_TOL)
    p.close()


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("fp32", None)])
def test_warp_local_rows_in_several_rounds(precision, tol):
    # nx = 128 (16 x 8): 16 threads per pencil, 16 pencils per round of 256
    # threads; in FP32 the strain passes hold 8 rows (24 pencils) per CTA, two
    # rounds; 60 rows in all, not a multiple of 8
    w = custom_workload((6, 10, 128), [0, 5], 2, seed=15, steps=3)
    p = Pair(w, precision, ms_tol=0.0, ms_max_it=4)
    p.run(3)
    e = p.errors()
    if tol is not None:
        check(e, tol)
    else:
        assert e["f_l2"] <= FP32_TOL and e["eps_l2"] <= FP32_TOL and e["sigma_l2"] <= FP32_TOL, e
    p.close()


@pytest.mark.parametrize("shape", [(20, 12, 16), (24, 24, 24)])
def test_fp32_fixed_passes(shape):
    vids = [0, 3] if shape[0] == 20 else [0, 1, 2, 3, 4, 5]
    w = custom_workload(shape, vids, 2 if shape[0] == 20 else 6, seed=15, eps_p=shape[0] == 20)
    p = Pair(w, "fp32", ms_tol=0.0, ms_max_it=8)
    p.run(4)
    e = p.errors()
    assert e["sigma_l2"] <= FP32_TOL and e["f_l2"] <= FP32_TOL and e["curve"] <= FP32_TOL, e
    p.close()


def test_fp32_converged_pillar_recipe():
    """The micro-pillar recipe (two variants, smooth plastic strain, ramp) at
    32^3: FP32 with tolerance 1e-6 against the oracle solved to 1e-12."""
    w = I.config2(steps=6, n=32, total_steps=20)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-6)
    o = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
    for k in range(6):
        code, info = h.step(w.E[k][None, None, :])
        assert code == pf.PF_OK and info[0].resid <= 1e-6
        oi = o.step(w.E[k])
        assert rel_max(np.array(info[0].mean_sigma[:]), oi["mean_sigma"]) <= FP32_TOL
    mean, sig = h.stress(0)
    f, eps = h.get_fields(0)
    so = O.tensor2_to_voigt(o.stress_field()).reshape(6, -1)
    assert rel_l2(sig, so) <= FP32_TOL
    assert rel_l2(f, o.f.reshape(2, -1)) <= FP32_TOL
    h.close()


def test_one_dimensional_interface_no_mechanics():
    # 64 x 1 x 1 grid: length-1 transforms along y and z
    n = 64
    x = np.arange(n)
    f = ((x >= 16) & (x < 48)).astype(np.float64)[None, None, None, :]
    E = np.zeros((50, 6))
    w = I.Workload("line", (1, 1, n), [0], f, None, None, np.eye(3)[None], E, twin_stiffness=0,
                   gamma_tw=0.0, dt=0.5, ms_tol=1e-12, precision="fp64")
    p = Pair(w, "fp64")
    p.run(50)
    e = p.errors()
    assert e["f_max"] <= FP64_TOL, e
    p.close()


def test_single_fourier_mode_closed_form_on_gpu():
    """Homogeneous HCP medium with eps* = eps0 cos(xi.x): eps = E + sym(a (x) xi)
    cos(xi.x) with K(xi) a = (C : eps0) xi, straight from equilibrium."""
    shape = (8, 10, 12)
    nz, ny, nx = shape
    m = np.array([2, -1, 3])
    xi = 2 * np.pi * m / np.array([nx, ny, nz])
    eps0 = O.voigt_to_tensor2(np.array([0.01, -0.004, 0.002, 0.003, -0.001, 0.005]))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cosx = np.cos(xi[0] * x + xi[1] * y + xi[2] * z)
    eps_p = O.tensor2_to_voigt(eps0[:, :, None, None, None] * cosx)
    E = np.array([[0.001, 0.0, -0.002, 0.0, 0.0005, 0.0]])
    w = I.Workload("mode", shape, [0], np.zeros((1,) + shape), eps_p, None, np.eye(3)[None], E,
                   twin_stiffness=0, ms_tol=1e-13, precision="fp64")
    h = pf.handle_for(w)
    h.step(E)
    _, eps = h.get_fields(0)
    C = O.voigt_to_tensor4(O.hcp_stiffness_voigt(*I.C_HEX_GPA))
    K = np.einsum("ijkl,j,l->ik", C, xi, xi)
    a = np.linalg.solve(K, np.einsum("ijkl,kl,j->i", C, eps0, xi))
    exact = O.voigt_to_tensor2(E[0])[..., None, None, None] + \
        (0.5 * (np.outer(a, xi) + np.outer(xi, a)))[..., None, None, None] * cosx
    assert rel_max(eps, O.tensor2_to_voigt(exact).reshape(6, -1)) <= 1e-12
    h.close()


def test_zero_stress_homogeneous_eigenstrain_gpu():
    shape = (8, 8, 8)
    f = np.full((1,) + shape, 0.4)
    tab = O.build_tables(I.C_HEX_GPA, I.C_OVER_A, [2], np.eye(3)[None], 1)
    E = 0.129 * 0.4 * O.tensor2_to_voigt(tab.S[0, 0])
    w = I.Workload("hom", shape, [2], f, None, None, np.eye(3)[None], E[None], ms_tol=1e-13,
                   precision="fp64")
    h = pf.handle_for(w)
    h.step(E[None, None, :])
    mean, sig = h.stress(0)
    assert np.abs(sig).max() <= 1e-13
    h.close()


def test_bitwise_reproducible_and_checkpoint_resume():
    w = custom_workload((16, 16, 16), [0, 3], 2, seed=21, steps=6)

    def run(split):
        h = pf.handle_for(w, precision="fp32", ms_tol=1e-6)
        for k in range(6):
            if k == split:
                f, eps = h.get_fields(0)
                h2 = pf.handle_for(w, precision="fp32", ms_tol=1e-6)
                N = w.nvox
                h2.set_fields(0, f, w.eps_p.reshape(6, N), w.grain.reshape(N), eps)
                h.close()
                h = h2
            h.step(w.E[k][None, None, :])
        out = h.get_fields(0)
        h.close()
        return out

    a = run(None)
    b = run(None)
    c = run(3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


def test_error_codes_noconv_and_nan():
    w = custom_workload((8, 8, 8), [0], 2, seed=22, steps=2)
    h = pf.handle_for(w, precision="fp32", ms_tol=1e-14, ms_max_it=2)
    code, info = h.step(w.E[:1][None], allow=(pf.PF_ENOCONV,))
    assert code == pf.PF_ENOCONV and info[0].status == pf.PF_ENOCONV and info[0].n_ms_last == 2
    h.close()
    bad = w.eps_p.copy()
    bad[0, 1, 2, 3] = np.nan
    w2 = I.Workload("nan", w.shape, w.variant_ids, w.f, bad, w.grain, w.grain_R, w.E)
    h = pf.handle_for(w2, precision="fp32", ms_tol=1e-6)
    code, info = h.step(w.E[:1][None], allow=(pf.PF_ENAN,))
    assert code == pf.PF_ENAN and info[0].status == pf.PF_ENAN
    h.close()


def test_device_memory_and_stream_match_host_path():
    torch = pytest.importorskip("torch")
    w = custom_workload((12, 16, 20), [1, 4], 2, seed=23, steps=3)
    N = w.nvox
    host = pf.handle_for(w, precision="fp32", ms_tol=1e-6)
    for k in range(3):
        host.step(w.E[k][None, None, :])
    fh, eh = host.get_fields(0)
    mh, sh = host.stress(0)
    host.close()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        cfg = pf.config_for(w, precision="fp32", ms_tol=1e-6, stream=s.cuda_stream)
        h = pf.Handle(cfg, 1, grain_R=w.grain_R)
        dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)
        fd = dev(w.f.reshape(2, N))
        ed = dev(w.eps_p.reshape(6, N))
        gd = torch.from_numpy(w.grain.reshape(N).astype(np.int16)).cuda()
        h.set_fields(0, fd, ed, gd, None, mem=pf.PF_MEM_DEVICE)
        for k in range(3):
            h.step(w.E[k][None, None, :])
        fo = torch.empty((2, N), device="cuda", dtype=torch.float32)
        eo = torch.empty((6, N), device="cuda", dtype=torch.float32)
        so = torch.empty((6, N), device="cuda", dtype=torch.float32)
        h.get_fields(0, fo, eo, mem=pf.PF_MEM_DEVICE)
        md, _ = h.stress(0, field=True, out=so, mem=pf.PF_MEM_DEVICE)
    s.synchronize()
    assert np.array_equal(fo.cpu().numpy(), fh) and np.array_equal(eo.cpu().numpy(), eh)
    assert np.array_equal(so.cpu().numpy(), sh) and np.array_equal(md, mh)
    h.close()


def test_invalid_arguments_on_gpu():
    cfg = pf.config_default()
    cfg.nx = 14  # 2 x 7
    with pytest.raises(pf.PfError):
        pf.Handle(cfg)
    w = custom_workload((8, 8, 8), [0], 2, seed=24, steps=1)
    h = pf.handle_for(w, precision="fp32")
    g = w.grain.reshape(-1).copy()
    g[5] = 7  # grain id beyond n_grains
    with pytest.raises(pf.PfError):
        h.set_fields(0, w.f.reshape(1, -1), None, g)
    h.close()


@pytest.mark.parametrize("level", [1, 2])
def test_discretisation_study_meshes(level):
    """The mesh1 / mesh2 grids of Sec. 6 (16x16x32, 32x32x64 cells): FP64
    within 1e-12 with fixed passes, the extrapolated warm start on."""
    w = I.mesh_study(level, steps=5)
    p = Pair(w, "fp64", ms_tol=0.0, ms_max_it=4, warm_degree=3)
    p.run(5)
    check(p.errors(), FP64_TOL)
    p.close()
