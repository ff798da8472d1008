"""Pins of the oracle's naive separable DFT against brute force and numpy.fft."""
import numpy as np
import pytest

from oracle import pf_oracle as O


def brute_force_dft3(a):
    """O(N^2) sum over every voxel for every mode, straight from the definition
    X(k) = sum_x a(x) exp(-2 pi i sum_j k_j x_j / n_j)."""
    nz, ny, nx = a.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([z.ravel(), y.ravel(), x.ravel()], axis=1)
    n = np.array([nz, ny, nx], dtype=np.float64)
    phase = (pos[:, None, :] * pos[None, :, :]) / n
    W = np.exp(-2j * np.pi * phase.sum(axis=-1))
    return (W @ a.ravel()).reshape(a.shape)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12), (5, 3, 7)])
def test_separable_dft_matches_brute_force(shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = brute_force_dft3(a)
    got = O.dft3(a)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 16, 64, 80, 96, 120, 128, 160])
def test_1d_dft_matches_numpy_fft(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    got = O.dft_axis(a, 1, -1.0)
    ref = np.fft.fft(a, axis=1)
    assert np.abs(got - ref).max() <= 1e-13 * n * np.abs(ref).max()


def test_round_trip_and_parseval():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 6, 10, 12))
    A = O.dft3(a)
    assert np.abs(O.idft3(A) - a).max() <= 1e-14 * 50
    # Parseval: sum |a|^2 = (1/N) sum |A|^2
    assert abs(np.sum(a * a) - np.sum(np.abs(A) ** 2) / a[0].size) <= 1e-12 * np.sum(a * a)


def test_real_input_spectrum_is_hermitian():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((6, 10, 12))
    A = O.dft3(a)
    # A(-k) = conj A(k)
    Am = np.roll(np.flip(A, axis=(0, 1, 2)), 1, axis=(0, 1, 2))
    assert np.abs(Am - np.conj(A)).max() <= 1e-12 * np.abs(A).max()


def test_wavevector_convention():
    (xx, yy, zz), nyq = O.wavevectors((4, 6, 5))
    # x: n = 5 (odd) -> m = 0, 1, 2, -2, -1 ; no Nyquist
    assert np.allclose(xx.ravel() * 5 / (2 * np.pi), [0, 1, 2, -2, -1])
    # y: n = 6 -> m = 0, 1, 2, -3, -2, -1 ; Nyquist index 3 maps to -n/2
    assert np.allclose(yy.ravel() * 6 / (2 * np.pi), [0, 1, 2, -3, -2, -1])
    assert nyq[0, 3, 0] and nyq[2, 0, 0] and not nyq[1, 1, 1]
