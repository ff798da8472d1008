"""Pins of the oracle's Green operator and Moulinec-Suquet solve against
closed forms and the equations of periodic elastic equilibrium."""
import math

import numpy as np
import pytest

from oracle import pf_oracle as O

C_A = 1.633
CHEX = (59.4, 25.6, 21.4, 61.6, 16.4)


def c_hcp():
    return O.voigt_to_tensor4(O.hcp_stiffness_voigt(*CHEX))


def test_green_projector_identities():
    """Gamma0 : C0 : Gamma0 = Gamma0, Gamma0 : C0 : sym(u (x) xi) = sym(u (x) xi),
    xi . (C0 : Gamma0 : tau) = xi . tau, and the minor/major symmetries."""
    rng = np.random.default_rng(5)
    R = O.axis_angle(rng.standard_normal(3), 1.1)
    C0 = O.rotate4(c_hcp(), R)
    xi = rng.standard_normal((20, 3))
    G = O.green_operator(C0, xi)
    GCG = np.einsum("mijab,abcd,mcdkl->mijkl", G, C0, G)
    assert np.abs(GCG - G).max() <= 1e-12 * np.abs(G).max()
    assert np.abs(G - G.transpose(0, 2, 1, 3, 4)).max() <= 1e-14 * np.abs(G).max()
    assert np.abs(G - G.transpose(0, 1, 2, 4, 3)).max() <= 1e-14 * np.abs(G).max()
    assert np.abs(G - G.transpose(0, 3, 4, 1, 2)).max() <= 1e-14 * np.abs(G).max()
    u = rng.standard_normal((20, 3))
    eps = 0.5 * (u[:, :, None] * xi[:, None, :] + xi[:, :, None] * u[:, None, :])
    back = np.einsum("mijab,abcd,mcd->mij", G, C0, eps)
    assert np.abs(back - eps).max() <= 1e-12 * np.abs(eps).max()
    tau = rng.standard_normal((20, 3, 3))
    tau = tau + tau.transpose(0, 2, 1)
    s = np.einsum("abcd,mcdkl,mkl->mab", C0, G, tau)
    assert np.abs(np.einsum("mij,mj->mi", s - tau, xi)).max() <= 1e-12 * np.abs(tau).max() * 3


def homogeneous_state(shape, f, eps_p, E, twin_stiffness=0, vids=(0,), gamma=0.129,
                      tol=1e-12, max_it=50):
    tab = O.build_tables(CHEX, C_A, list(vids), np.eye(3)[None], twin_stiffness)
    p = O.Params(0.03125, 0.0176, 1.0, 0.05, gamma, tol, max_it)
    return O.State(f, eps_p, None, tab, p), tab


def test_ms_homogeneous_converges_in_one_pass():
    shape = (6, 8, 10)
    rng = np.random.default_rng(0)
    f = rng.random((1,) + shape)
    E = np.array([-0.003, 0.001, 0.002, 0.0005, -0.0002, 0.0007])
    st, tab = homogeneous_state(shape, f, None, E)
    C0 = O.mean_stiffness(st.f, None, tab)
    start = np.broadcast_to(O.voigt_to_tensor2(E)[..., None, None, None], (3, 3) + shape).copy()
    eps1, n1, r1 = O.ms_solve(st.f, None, None, tab, 0.129, C0, E, start, 0.0, 1)
    eps2, n2, r2 = O.ms_solve(st.f, None, None, tab, 0.129, C0, E, eps1, 0.0, 1)
    assert r2 <= 1e-14


def test_single_fourier_mode_closed_form():
    """Homogeneous HCP medium, eps* = eps0 cos(xi . x): the displacement
    amplitude a solves K(xi) a = (C : eps0) xi, so eps = E + sym(a (x) xi) cos(xi.x)."""
    shape = (8, 10, 12)
    nz, ny, nx = shape
    m = np.array([2, -1, 3])  # mode numbers along x, y, z
    xi = 2 * np.pi * m / np.array([nx, ny, nz])
    eps0 = O.voigt_to_tensor2(np.array([0.01, -0.004, 0.002, 0.003, -0.001, 0.005]))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cosx = np.cos(xi[0] * x + xi[1] * y + xi[2] * z)
    eps_p = O.tensor2_to_voigt(eps0[:, :, None, None, None] * cosx)
    E = np.array([0.001, 0.0, -0.002, 0.0, 0.0005, 0.0])
    st, tab = homogeneous_state(shape, np.zeros((1,) + shape), eps_p, E)
    st.step(E)
    C = c_hcp()
    K = np.einsum("ijkl,j,l->ik", C, xi, xi)
    a = np.linalg.solve(K, np.einsum("ijkl,kl,j->i", C, eps0, xi))
    exact = O.voigt_to_tensor2(E)[..., None, None, None] + \
        (0.5 * (np.outer(a, xi) + np.outer(xi, a)))[..., None, None, None] * cosx
    assert np.abs(st.eps - exact).max() <= 1e-12 * np.abs(exact).max()
    sig = st.stress_field()
    sh = O.dft3(sig)
    xi_all, _ = O.wavevectors(shape)
    div = sum(sh[:, j] * xi_all[j] for j in range(3))
    assert np.abs(div).max() <= 1e-10 * np.abs(sh).max()


def test_zero_stress_for_homogeneous_eigenstrain():
    shape = (6, 6, 8)
    f = np.full((1,) + shape, 0.37)
    ep = np.zeros((6,) + shape)
    ep[:] = np.array([0.001, -0.002, 0.001, 0.0003, 0.0, -0.0004])[:, None, None, None]
    tab = O.build_tables(CHEX, C_A, [2], np.eye(3)[None], 1)
    estar = O.eigenstrain(f, ep, None, tab, 0.129)
    E = O.tensor2_to_voigt(estar[:, :, 0, 0, 0])
    st = O.State(f, ep, None, tab, O.Params(0.03125, 0.0176, 1.0, 0.05, 0.129, 1e-12, 20))
    st.step(E)
    assert np.abs(st.stress_field()).max() <= 1e-14


def test_mean_stress_homogeneous_medium():
    """<sigma> = C : (E - <eps*>) exactly when C is uniform."""
    shape = (8, 8, 8)
    rng = np.random.default_rng(2)
    f = rng.random((1,) + shape) * 0.8
    ep = rng.standard_normal((6,) + shape) * 1e-3
    E = np.array([-0.004, 0.001, 0.0, 0.0, 0.001, 0.0])
    st, tab = homogeneous_state(shape, f, ep, E)
    estar_mean = O.eigenstrain(st.f, ep, None, tab, 0.129).mean(axis=(2, 3, 4))
    info = st.step(E)
    expect = O.tensor2_to_voigt(np.einsum("ijkl,kl->ij", c_hcp(), O.voigt_to_tensor2(E) - estar_mean))
    assert np.abs(info["mean_sigma"] - expect).max() <= 1e-12 * np.abs(expect).max()


def _heterogeneous_case(shape, seed=7):
    rng = np.random.default_rng(seed)
    f = np.zeros((2,) + shape)
    f[0] = (rng.random(shape) < 0.3) * 1.0
    f[1] = (1 - f[0]) * (rng.random(shape) < 0.2)
    grain = (rng.random(shape) < 0.5).astype(np.uint16)
    R = np.stack([np.eye(3), O.axis_angle([0.3, -1.0, 0.4], 1.3)])
    tab = O.build_tables(CHEX, C_A, [0, 3], R, 1)
    ep = rng.standard_normal((6,) + shape) * 1e-3
    return f, grain, tab, ep


def test_heterogeneous_solution_is_equilibrated_and_compatible():
    """With rotated twin stiffness and two grains the converged field must
    satisfy xi . sigma_hat = 0 (equilibrium), the Saint-Venant compatibility
    eps_ikl eps_jmn xi_k xi_m eps_hat_ln = 0, and <eps> = E.  Odd grid sizes
    have no Nyquist modes, so these hold at every mode."""
    shape = (5, 7, 9)
    f, grain, tab, ep = _heterogeneous_case(shape)
    E = np.array([-0.005, 0.002, 0.001, 0.0, 0.001, -0.001])
    p = O.Params(0.03125, 0.0176, 1.0, 0.05, 0.129, 1e-14, 500)
    st = O.State(f, ep, grain, tab, p)
    info = st.step(E)
    assert info["n_ms"] < 500
    sh = O.dft3(st.stress_field())
    xi, _ = O.wavevectors(shape)
    div = sum(sh[:, j] * xi[j] for j in range(3))
    assert np.abs(div).max() <= 1e-11 * np.abs(sh).max()
    eh = O.dft3(st.eps)
    lc = np.zeros((3, 3, 3))
    lc[0, 1, 2] = lc[1, 2, 0] = lc[2, 0, 1] = 1
    lc[0, 2, 1] = lc[2, 1, 0] = lc[1, 0, 2] = -1
    xib = [np.broadcast_to(x, shape) for x in xi]
    inc = np.zeros((3, 3) + shape, dtype=complex)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    for m in range(3):
                        for n in range(3):
                            c = lc[i, k, l] * lc[j, m, n]
                            if c:
                                inc[i, j] += c * xib[k] * xib[m] * eh[l, n]
    assert np.abs(inc).max() <= 1e-11 * np.abs(eh[:, :, 1:]).max()
    assert np.allclose(st.eps.mean(axis=(2, 3, 4)), O.voigt_to_tensor2(E), atol=1e-15)


def test_ms_residual_contracts_and_iteration_count():
    shape = (6, 6, 6)
    f, grain, tab, ep = _heterogeneous_case(shape, seed=3)
    E = np.array([-0.005, 0.0, 0.0, 0.0, 0.0, 0.0])
    C0 = O.mean_stiffness(f, grain, tab)
    start = np.broadcast_to(O.voigt_to_tensor2(E)[..., None, None, None], (3, 3) + shape).copy()
    res = []
    eps = start
    for _ in range(6):
        eps, _, r = O.ms_solve(f, ep, grain, tab, 0.129, C0, E, eps, 0.0, 1)
        res.append(r)
    assert all(res[i + 1] < res[i] for i in range(len(res) - 1))
    _, n, r = O.ms_solve(f, ep, grain, tab, 0.129, C0, E, start, 1e-6, 100)
    assert r <= 1e-6 and n < 100


def test_periodic_shift_equivariance():
    """Shifting every input field by an integer periodic offset shifts every
    output of a full step (solve + update) by the same offset."""
    shape = (6, 8, 10)
    f, grain, tab, ep = _heterogeneous_case(shape, seed=11)
    f = f * 0.7
    E = np.array([-0.004, 0.001, 0.0, 0.0, 0.0005, 0.0])
    p = O.Params(0.03125, 0.0176, 1.0, 0.05, 0.129, 0.0, 8)
    sh = (1, -3, 4)
    ax = (-3, -2, -1)
    a = O.State(f, ep, grain, tab, p)
    b = O.State(np.roll(f, sh, ax), np.roll(ep, sh, ax), np.roll(grain, sh, ax), tab, p)
    a.step(E)
    b.step(E)
    assert np.abs(np.roll(a.f, sh, ax) - b.f).max() <= 1e-12
    assert np.abs(np.roll(a.eps, sh, ax) - b.eps).max() <= 1e-12 * np.abs(a.eps).max()
