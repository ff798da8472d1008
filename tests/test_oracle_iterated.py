"""Pins of the iterated step (reading R12 of the oracle): one pass is the
semi-implicit step, the converged i-loop solves the fully implicit step, its
fixed point is that of the paper's literal linearised equation (Eq. fRate3
with the variable coefficient, solved densely on a small 1-D grid), and the
j-loop projection."""
import math

import numpy as np

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I

C_A = 1.633
CHEX = (59.4, 25.6, 21.4, 61.6, 16.4)
C1 = 0.03125


def small_crystal(steps=2):
    rng = np.random.Generator(np.random.PCG64(21))
    shape = (6, 8, 10)
    R = I.shoemake_rotations(rng, 1)
    f = 0.3 * rng.random((2,) + shape)
    E = np.stack([I.uniaxial_strain(-0.01, (0.0, 0.0, 1.0))] * steps)
    return I.Workload("crystal", shape, [0, 3], f, None, None, R, E)


def test_one_pass_is_the_semi_implicit_step():
    w = small_crystal()
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=100)
    b = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=100, n_pic=1)
    a.step(w.E[0])
    b.step(w.E[0])
    assert np.array_equal(a.f, b.f)


def test_converged_loop_is_the_implicit_step():
    """(f - f^n)/dt = c3 (c2 lap f + d(f)) at the strain of the step."""
    w = small_crystal()
    st = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=100, n_pic=60)
    info = st.step(w.E[0])
    assert info["pic_change"] <= 1e-14
    d, _ = O.driving_force(st.f, st.eps, None, None, st.tab, w.c1, w.gamma_tw)
    k2 = O.laplace_symbol(w.shape)
    for a in range(w.V):
        lap = O.idft3(-k2 * O.dft3(st.f[a])).real
        res = (st.f[a] - st.f_solved[a]) / w.dt - w.c3 * (w.c2 * lap + d[a])
        assert np.abs(res).max() <= 1e-11 * np.abs(d[a]).max()


def test_fixed_point_of_the_literal_linearised_equation():
    """One variant, no mechanics, 1-D: iterate the printed form
    f^i/dt - c3 c2 [sum_{b != a} f_b^(i-1)] lap f^i + r^i = 0 (dense solve,
    variable coefficient, r^i with its c3 c2 f_a lap f_b term) to its fixed
    point and compare with the R12 loop's."""
    n, c2, c3, dt = 16, 0.04, 1.0, 2.0
    x = np.arange(n)
    f_n = 0.5 + 0.4 * np.cos(2 * np.pi * x / n) + 0.05 * np.sin(6 * np.pi * x / n)
    F = np.fft.fft(np.eye(n), axis=0)
    k = np.fft.fftfreq(n) * 2 * np.pi
    D2 = np.real(np.linalg.inv(F) @ np.diag(-k * k) @ F)  # spectral Laplacian as a matrix
    f = f_n.copy()
    for _ in range(400):
        f0 = 1.0 - f  # the matrix phase, the only other phase
        chem = f * f0 * (f0 - f)  # sum_b f_a f_b (f_b - f_a)
        r = -f_n / dt + c3 * C1 * chem + c3 * c2 * f * (D2 @ f0)
        Amat = np.eye(n) / dt - c3 * c2 * np.diag(f0) @ D2
        f_new = np.linalg.solve(Amat, -r)
        if np.abs(f_new - f).max() < 1e-15:
            break
        f = f_new
    # the R12 loop on the same problem
    tab = O.build_tables(CHEX, C_A, [0], np.eye(3)[None], 0)
    p = O.Params(C1, c2, c3, dt, 0.0, 1e-12, 5, True, n_pic=400)
    st = O.State(f_n[None, None, None, :], None, None, tab, p)
    st.step(np.zeros(6))
    assert np.abs(st.f[0, 0, 0] - f).max() <= 1e-10


def test_projection():
    rng = np.random.default_rng(5)
    f = rng.uniform(-0.3, 1.3, (3, 4, 5, 6))
    g = O.clamp_phases(f)
    assert g.min() >= 0.0 and g.max() <= 1.0
    assert g.sum(axis=0).max() <= 1.0 + 1e-15
    ok = np.clip(f, 0, 1)
    s = ok.sum(axis=0)
    inside = s <= 1.0
    assert np.array_equal(g[:, inside], ok[:, inside])  # admissible points untouched after clipping
    out = ~inside
    ratio = g[:, out] / np.where(ok[:, out] > 0, ok[:, out], 1.0)
    assert np.allclose(ratio[ok[:, out] > 0], np.broadcast_to(1.0 / s[out], ratio.shape)[ok[:, out] > 0])
