"""Pins of the anisotropic gradient coefficient (reading R10 of the oracle,
Table 5's c2 along the twin-plane normal and along the shear direction):
the tensor's eigenpairs, the isotropic special case, the closed-form
gradient energy of a plane wave, a real and even operator on even grids, and
the relaxed 1-D interface width along the normal and along the shear
direction."""
import math

import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_2302_13612_gb300 import inputs as I

C_A = 1.633
CHEX = (59.4, 25.6, 21.4, 61.6, 16.4)
C1 = 0.03125


def rotation_onto_x(u):
    """A rotation R with R u = e_x (Rodrigues about u x e_x)."""
    u = u / np.linalg.norm(u)
    ex = np.array([1.0, 0.0, 0.0])
    ax = np.cross(u, ex)
    if np.linalg.norm(ax) < 1e-14:
        return np.eye(3) if u[0] > 0 else np.diag([-1.0, -1.0, 1.0])
    ang = math.acos(np.clip(np.dot(u, ex), -1.0, 1.0))
    return O.axis_angle(ax, ang)


def test_gradient_tensor_eigenpairs():
    rng = np.random.Generator(np.random.PCG64(5))
    R = I.shoemake_rotations(rng, 1)[0]
    c2 = (0.1, 0.7, 0.4)
    A = O.gradient_tensors(range(6), C_A, R, c2)
    for v in range(6):
        s, m = O.twin_system(v, C_A)
        n, sv = R @ m, R @ s
        t = np.cross(n, sv)
        assert abs(np.dot(n, sv)) < 1e-12  # the shear direction lies in the plane
        for vec, lam in ((n, c2[0]), (sv, c2[1]), (t, c2[2])):
            assert np.allclose(A[v] @ vec, lam * vec, atol=1e-14)
        assert np.allclose(A[v], A[v].T, atol=1e-15)


def test_isotropic_special_case():
    rng = np.random.default_rng(3)
    f = rng.random((2, 6, 5, 8))
    d = rng.standard_normal((2, 6, 5, 8))
    c2 = 0.021
    A = np.array([c2 * np.eye(3)] * 2)
    a = O.allen_cahn_update(f, d, c2, 1.3, 0.4)
    b = O.allen_cahn_update(f, d, c2, 1.3, 0.4, A)
    assert np.abs(a - b).max() <= 1e-14
    tab = O.build_tables(CHEX, C_A, [0, 3], np.eye(3)[None], 1)
    eps = np.zeros((3, 3) + f.shape[1:])
    ga = O.energy_parts(f, eps, None, None, tab, C1, c2, 0.129)
    gb = O.energy_parts(f, eps, None, None, tab, C1, c2, 0.129, A)
    assert abs(ga[2] - gb[2]) <= 1e-13 * abs(ga[2])


def test_plane_wave_gradient_energy():
    """f = a cos(xi.x): sum_x 1/2 grad f . A grad f = N a^2 (xi.A.xi) / 4."""
    shape = (10, 6, 8)
    nz, ny, nx = shape
    m = (1, 2, -1)  # (x, y, z) wave numbers, none at the Nyquist index
    xi = 2 * np.pi * np.array([m[0] / nx, m[1] / ny, m[2] / nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    amp = 0.3
    f = (amp * np.cos(xi[0] * x + xi[1] * y + xi[2] * z))[None]
    rng = np.random.Generator(np.random.PCG64(9))
    R = I.shoemake_rotations(rng, 1)[0]
    A = O.gradient_tensors([2], C_A, R, (0.05, 0.5, 0.2))
    tab = O.build_tables(CHEX, C_A, [2], R[None], 1)
    eps = np.zeros((3, 3) + shape)
    g_gd = O.energy_parts(f, eps, None, None, tab, C1, 0.0, 0.0, A)[2]
    expect = f[0].size * amp ** 2 * float(xi @ A[0] @ xi) / 4.0
    assert abs(g_gd - expect) <= 1e-12 * expect


def test_operator_is_real_on_even_grids():
    """Dropping the Nyquist cross terms keeps the update of a real field real."""
    rng = np.random.default_rng(4)
    shape = (6, 8, 4)
    f = rng.random((1,) + shape)
    R = I.shoemake_rotations(np.random.Generator(np.random.PCG64(2)), 1)[0]
    A = O.gradient_tensors([1], C_A, R, (0.2, 2.0, 1.0))
    den = 1.0 + 0.7 * O.gradient_symbol(shape, A[0])
    out = O.idft3(O.dft3(f[0]) / den)
    assert np.abs(out.imag).max() <= 1e-14 * np.abs(out.real).max()
    # and symmetric under xi -> -xi (index k -> -k mod n on every axis)
    flip = den[np.ix_(*[(-np.arange(n)) % n for n in shape])]
    assert np.array_equal(den, flip)


def relaxed_width(c2_nst, align, n, steps):
    """1-D run along x of variant 0 with its normal (align='n') or shear
    direction (align='s') turned onto x; returns the fitted width W = 4w."""
    s, m = O.twin_system(0, C_A)
    R = rotation_onto_x(m if align == "n" else s)
    A = O.gradient_tensors([0], C_A, R, c2_nst)
    tab = O.build_tables(CHEX, C_A, [0], R[None], 0)
    x = np.arange(n)
    f = ((x >= n // 4) & (x < 3 * n // 4)).astype(np.float64)[None, None, None, :]
    p = O.Params(C1, 0.0, 1.0, 1.0, 0.0, 1e-12, 5, True, A)
    st = O.State(f, None, None, tab, p)
    for _ in range(steps):
        st.step(np.zeros(6))
    fr = st.f[0, 0, 0]
    i = np.argmax((fr[:-1] < 0.5) & (fr[1:] >= 0.5))
    x0 = i + (0.5 - fr[i]) / (fr[i + 1] - fr[i])
    half = slice(0, n // 2)
    best = (np.inf, None)
    for w in np.linspace(0.3, 2.5, 441):
        for dx in np.linspace(-0.02, 0.02, 11):
            r = np.sum((fr[half] - 0.5 * (1 + np.tanh((x[half] - x0 - dx) / (2 * w)))) ** 2)
            if r < best[0]:
                best = (r, w)
    return 4 * best[1]


@pytest.mark.parametrize("align,W", [("n", 3.0), ("s", 6.0)])
def test_interface_width_follows_the_direction(align, W):
    """c2_n = c1 (3/4)^2 and c2_s = c2_t = 4 c2_n: the interface whose normal is
    the twin-plane normal is 3 voxels wide, one whose normal is the shear
    direction 6 voxels (W = 4 sqrt(c2/c1), reading R2)."""
    c2n = C1 * 0.75 ** 2
    Wfit = relaxed_width((c2n, 4 * c2n, 4 * c2n), align, n=128, steps=2500 if align == "s" else 1500)
    assert abs(Wfit - W) / W < 0.02, Wfit
