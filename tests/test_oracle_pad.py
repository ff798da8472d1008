"""Pins of the pad-layer mobility (reading R11 of the oracle): unit mobility
reproduces the plain update, the converged corrections solve the
variable-mobility semi-implicit equation, a zero-mobility pad keeps its
order parameter, and the corrections contract."""
import numpy as np

from oracle import pf_oracle as O

C2, C3, DT = 0.02, 1.0, 0.5


def fields(shape=(6, 8, 10), V=2, seed=1):
    rng = np.random.default_rng(seed)
    f = rng.random((V,) + shape) * 0.5
    d = rng.standard_normal((V,) + shape) * 0.1
    return f, d


def pad_mask(shape, w=2, low=0.0):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pad = (x < w) | (x >= nx - w) | (y < w) | (y >= ny - w)
    return np.where(pad, low, 1.0), pad


def test_unit_mobility_is_the_plain_update():
    f, d = fields()
    a = O.allen_cahn_update(f, d, C2, C3, DT)
    b, change = O.allen_cahn_update(f, d, C2, C3, DT, M=np.ones(f.shape[1:]), n_corr=3)
    assert np.abs(a - b).max() <= 1e-14
    assert change <= 1e-15


def test_converged_corrections_solve_the_equation():
    """(f' - f)/dt = c3 M (c2 lap f' + d) once the corrections have converged."""
    f, d = fields()
    M, _ = pad_mask(f.shape[1:], low=0.05)
    out, change = O.allen_cahn_update(f, d, C2, C3, DT, M=M, n_corr=40)
    assert change <= 1e-14
    k2 = O.laplace_symbol(f.shape[1:])
    for a in range(f.shape[0]):
        lap = O.idft3(-k2 * O.dft3(out[a])).real
        res = (out[a] - f[a]) / DT - C3 * M * (C2 * lap + d[a])
        assert np.abs(res).max() <= 1e-12 * np.abs(d[a]).max()


def test_zero_mobility_pad_keeps_f():
    f, d = fields(seed=2)
    M, pad = pad_mask(f.shape[1:], low=0.0)
    out, _ = O.allen_cahn_update(f, d, C2, C3, DT, M=M, n_corr=40)
    assert np.abs(out[:, pad] - f[:, pad]).max() <= 1e-12
    assert np.abs(out[:, ~pad] - f[:, ~pad]).max() > 1e-3  # the sample itself evolves


def test_corrections_contract():
    f, d = fields(seed=3)
    M, _ = pad_mask(f.shape[1:], low=0.01)
    changes = [O.allen_cahn_update(f, d, C2, C3, DT, M=M, n_corr=k)[1] for k in range(1, 6)]
    assert all(b < 0.5 * a for a, b in zip(changes, changes[1:])), changes
