"""Pins of the extrapolated warm start (reading R9 of the oracle): the
extrapolation is exact on polynomial histories of its degree, the converged
strain does not depend on the start, and a smooth run needs fewer passes as
the degree grows."""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I


def test_extrapolation_exact_on_polynomials():
    rng = np.random.default_rng(7)
    A, B, C, D = (rng.standard_normal((3, 3, 4, 5, 6)) for _ in range(4))
    cub = [A + B * k + C * k * k + D * k ** 3 for k in range(5)]
    assert np.allclose(O.extrapolate_start(cub[:4]), cub[4], rtol=0, atol=1e-11)
    quad = [A + B * k + C * k * k for k in range(4)]
    assert np.allclose(O.extrapolate_start(quad[:3]), quad[3], rtol=0, atol=1e-12)
    lin = [A + B * k for k in range(3)]
    assert np.allclose(O.extrapolate_start(lin[:2]), lin[2], rtol=0, atol=1e-13)
    assert np.array_equal(O.extrapolate_start([A]), A)
    # one degree short misses by the next backward difference: 2C for a quadratic
    # seen through the linear rule, 6D for a cubic seen through the quadratic rule
    assert np.allclose(O.extrapolate_start(quad[1:3]) - quad[3], -2 * C, atol=1e-12)
    assert np.allclose(O.extrapolate_start(cub[1:4]) - cub[4], -6 * D, atol=1e-11)


def test_coefficients_are_the_backward_difference_weights():
    e = [np.array([float(100 ** k)]) for k in range(6)]  # digit pairs expose each weight
    assert O.extrapolate_start(e[:2])[0] == 2 * 100 - 1
    assert O.extrapolate_start(e[:3])[0] == 3 * 100 ** 2 - 3 * 100 + 1
    assert O.extrapolate_start(e[:4])[0] == 4 * 100 ** 3 - 6 * 100 ** 2 + 4 * 100 - 1
    assert O.extrapolate_start(e[:5])[0] == 5 * 100 ** 4 - 10 * 100 ** 3 + 10 * 100 ** 2 - 5 * 100 + 1
    assert O.extrapolate_start(e[:6])[0] == (6 * 100 ** 5 - 15 * 100 ** 4 + 20 * 100 ** 3 - 15 * 100 ** 2
                                             + 6 * 100 - 1)


def test_exact_on_quintic_history():
    rng = np.random.default_rng(8)
    c = [rng.standard_normal((3, 3, 2, 3, 4)) for _ in range(6)]
    seq = [sum(ci * float(k) ** i for i, ci in enumerate(c)) for k in range(7)]
    assert np.allclose(O.extrapolate_start(seq[:6]), seq[6], rtol=1e-9, atol=1e-8)
    quart = [sum(ci * float(k) ** i for i, ci in enumerate(c[:5])) for k in range(6)]
    assert np.allclose(O.extrapolate_start(quart[:5]), quart[5], rtol=1e-10, atol=1e-9)


def small_poly(steps=6, n=16):
    return I.config3(steps=steps, n=n, seed=1003, n_grains=4)


@pytest.mark.parametrize("degree", [2, 3])
def test_converged_strain_independent_of_start(degree):
    w = small_poly(6)
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
    b = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm_degree=degree)
    for k in range(6):
        a.step(w.E[k])
        b.step(w.E[k])
        d = np.abs(a.eps - b.eps).max() / np.abs(a.eps).max()
        assert d <= 1e-10, (k, d)
    assert np.abs(a.f - b.f).max() <= 1e-10


def test_smooth_run_needs_fewer_passes():
    w = small_poly(9)
    tot = {}
    for d in (0, 1, 2, 3):
        st = O.state_from_workload(w, ms_tol=1e-8, ms_max_it=200, warm_degree=d)
        tot[d] = [st.step(w.E[k])["n_ms"] for k in range(9)]
    # identical while one solution is held, then fewer passes with each degree
    assert len({t[0] for t in tot.values()}) == 1 and len({t[1] for t in tot.values()}) == 1
    late = {d: sum(t[5:]) for d, t in tot.items()}
    assert late[3] < late[2] < late[1] < late[0], tot


def test_given_strain_counts_as_one_solution():
    w = small_poly(3)
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200)
    a.step(w.E[0])
    eps1 = a.eps_voigt()
    b = O.state_from_workload(w, ms_tol=0.0, ms_max_it=3, eps0=eps1, warm_degree=3)
    c = O.state_from_workload(w, ms_tol=0.0, ms_max_it=3, eps0=eps1)
    # with one held solution the start is that solution: same iterates as the plain warm start
    b.step(w.E[1])
    c.step(w.E[1])
    assert np.array_equal(b.eps, c.eps)
    assert len(b.sols) == 2


# ---- least-squares form (warm_points > warm_degree + 1) ----------------------
def test_least_squares_weights_closed_forms():
    from fractions import Fraction as Fr

    def exact(m, d):
        # the fitted polynomial's value at t = 1 as weights over the values at
        # t = 0, -1, ..., -(m-1): solve the normal equations (V^T V) c = V^T y
        # in exact rationals for each unit data vector y
        t = [Fr(-i) for i in range(m)]
        V = [[ti ** j for j in range(d + 1)] for ti in t]
        out = []
        for k in range(m):
            A = [[sum(V[i][r] * V[i][c] for i in range(m)) for c in range(d + 1)] for r in range(d + 1)]
            b = [V[k][r] for r in range(d + 1)]
            for col in range(d + 1):  # Gauss-Jordan
                piv = A[col][col]
                A[col] = [x / piv for x in A[col]]
                b[col] /= piv
                for r in range(d + 1):
                    if r != col and A[r][col] != 0:
                        f = A[r][col]
                        A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                        b[r] -= f * b[col]
            out.append(sum(b))  # sum_j c_j 1^j
        return out

    # the regression line through three points: 4/3, 1/3, -2/3
    assert exact(3, 1) == [Fr(4, 3), Fr(1, 3), Fr(-2, 3)]
    for m, d in [(3, 1), (4, 1), (4, 2), (5, 2), (5, 3), (6, 2), (6, 3), (6, 4)]:
        w = O.extrapolate_weights(m, d)
        assert np.allclose(w, [float(x) for x in exact(m, d)], rtol=0, atol=1e-12), (m, d)


@pytest.mark.parametrize("m,d", [(4, 2), (5, 2), (6, 3), (5, 3), (6, 2)])
def test_least_squares_exact_on_polynomials_of_its_degree(m, d):
    rng = np.random.default_rng(9)
    c = [rng.standard_normal((3, 3, 2, 3, 4)) for _ in range(d + 1)]
    seq = [sum(ci * float(k) ** i for i, ci in enumerate(c)) for k in range(m + 1)]
    assert np.allclose(O.extrapolate_start(seq[:m], d), seq[m], rtol=1e-10, atol=1e-9)


def test_least_squares_reduces_to_interpolation_and_damps_noise():
    rng = np.random.default_rng(10)
    s = [rng.standard_normal((3, 3, 2, 2, 2)) for _ in range(4)]
    # as many solutions as the degree needs: the interpolation weights
    assert np.array_equal(O.extrapolate_start(s, 3), O.extrapolate_start(s))
    # the same order of accuracy with a smaller weight norm (less amplified
    # rounding of the held solutions) when more solutions are held
    for d in (1, 2, 3):
        for m in range(d + 2, 7):
            assert np.linalg.norm(O.extrapolate_weights(m, d)) < np.linalg.norm(O.extrapolate_weights(d + 1)), (m, d)
        # exact on degree >= 1: sum_i w_i = 1 and sum_i w_i t_i = 1 at t_i = -i
        w = O.extrapolate_weights(6, d)
        assert abs(w.sum() - 1) < 1e-12 and abs((w * -np.arange(6)).sum() - 1) < 1e-12


def test_least_squares_state_holds_more_solutions():
    w = small_poly(8)
    a = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm_degree=2)
    b = O.state_from_workload(w, ms_tol=1e-12, ms_max_it=200, warm_degree=2, warm_points=5)
    for k in range(8):
        a.step(w.E[k])
        b.step(w.E[k])
        assert len(b.sols) == min(k + 1, 5) and len(a.sols) == min(k + 1, 3)
        # the converged strain does not depend on the start
        assert np.abs(a.eps - b.eps).max() <= 1e-10 * np.abs(a.eps).max(), k
