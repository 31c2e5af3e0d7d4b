"""Pins of the oracle's radix-2 FFT (the transforms of Sec. 3.3 / Eq. 11)
against the O(N^2) definition of the DFT, Parseval and the round trip."""
import numpy as np
import pytest

import oracle


def dft_matrix(n, sign):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256])
def test_fft1d_matches_direct_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dft_matrix(n, -1) @ x
    got = oracle.fft1d(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    inv = oracle.fft1d(ref, inverse=True)
    assert np.max(np.abs(inv - x)) <= 1e-13 * max(1.0, np.max(np.abs(x)))


def test_fft1d_parseval():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    X = oracle.fft1d(x)
    assert abs(np.sum(np.abs(X) ** 2) / 512 - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)


@pytest.mark.parametrize("ny,nx", [(4, 8), (8, 16), (2, 32)])
def test_fft2d_matches_direct_dft(ny, nx):
    rng = np.random.default_rng(nx * ny)
    x = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    ref = dft_matrix(ny, -1) @ x @ dft_matrix(nx, -1).T
    got = oracle.fft2d(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = oracle.fft2d(got, inverse=True)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))


def test_fft2d_threads_identical():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 64)) + 1j * rng.standard_normal((16, 64))
    a = oracle.fft2d(x, threads=False)
    b = oracle.fft2d(x, threads=True)
    assert np.array_equal(a, b)
