"""Pins of the extrapolated warm start (reading R9 of the oracle): the
extrapolation is exact on polynomial histories of its order, the converged
strain does not depend on the start, and a smooth run needs fewer passes."""
import numpy as np

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I


def test_extrapolation_exact_on_polynomials():
    rng = np.random.default_rng(7)
    A, B, C = (rng.standard_normal((3, 3, 4, 5, 6)) for _ in range(3))
    s = [A + B * k + C * k * k for k in range(4)]
    assert np.allclose(O.extrapolate_start(s[:3]), s[3], rtol=0, atol=1e-12)
    lin = [A + B * k for k in range(3)]
    assert np.allclose(O.extrapolate_start(lin[:2]), lin[2], rtol=0, atol=1e-13)
    assert np.array_equal(O.extrapolate_start([A]), A)
    # a quadratic history seen through the linear rule misses by the second difference 2C
    assert np.allclose(O.extrapolate_start(s[1:3]) - s[3], -2 * C, atol=1e-12)


def small_poly(steps=6, n=16):
    return I.config3(steps=steps, n=n, seed=1003, n_grains=4)


def test_converged_strain_independent_of_start():
    w = small_poly(5)
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
    b = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm="extrapolate")
    for k in range(5):
        a.step(w.E[k])
        b.step(w.E[k])
        d = np.abs(a.eps - b.eps).max() / np.abs(a.eps).max()
        assert d <= 1e-10, (k, d)
    assert np.abs(a.f - b.f).max() <= 1e-10


def test_smooth_run_needs_fewer_passes():
    w = small_poly(8)
    tot = {}
    for warm in ("previous", "extrapolate"):
        st = O.state_from_workload(w, ms_tol=1e-8, ms_max_it=200, warm=warm)
        tot[warm] = [st.step(w.E[k])["n_ms"] for k in range(8)]
    # identical until three solutions are held, then strictly fewer passes
    assert tot["previous"][:2] == tot["extrapolate"][:2]
    assert sum(tot["extrapolate"][3:]) < sum(tot["previous"][3:]), tot


def test_given_strain_counts_as_one_solution():
    w = small_poly(3)
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
    a.step(w.E[0])
    eps1 = a.eps_voigt()
    b = O.state_from_workload(w, ms_tol=0.0, ms_max_it=3, eps0=eps1, warm="extrapolate")
    c = O.state_from_workload(w, ms_tol=0.0, ms_max_it=3, eps0=eps1)
    # with one held solution the start is that solution: same iterates as the plain warm start
    b.step(w.E[1])
    c.step(w.E[1])
    assert np.array_equal(b.eps, c.eps)
    assert len(b.sols) == 2
