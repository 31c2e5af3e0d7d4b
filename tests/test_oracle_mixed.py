"""Pins of the oracle on grids whose sizes are not powers of two (the paper's
grids have 7 * 2^k points in tau and 1250 * 2^k in y, Table 1): the
mixed-radix transforms against the O(N^2) definition of the DFT, Parseval and
the round trip; the whole step against the closed form of a propagating
Fourier mode and against conservation of the mean."""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs


def dft_matrix(n, sign):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(k, k) % n) / n)


@pytest.mark.parametrize("n", [3, 5, 6, 7, 10, 12, 14, 25, 28, 49, 50, 56, 112, 125, 250, 448])
def test_fft1d_matches_direct_dft(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = dft_matrix(n, -1) @ x
    got = oracle.fft1d(x)
    assert np.max(np.abs(got - ref)) <= 2e-13 * max(1.0, np.max(np.abs(ref)))
    inv = oracle.fft1d(ref, inverse=True)
    assert np.max(np.abs(inv - x)) <= 2e-13 * max(1.0, np.max(np.abs(x)))


@pytest.mark.parametrize("n", [1250, 1792, 3584])
def test_fft1d_paper_lengths_parseval_and_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = oracle.fft1d(x)
    e = np.sum(np.abs(x) ** 2)
    assert abs(np.sum(np.abs(X) ** 2) / n - e) < 1e-12 * e
    # an independent library transform
    assert np.max(np.abs(X - np.fft.fft(x))) < 1e-11 * np.max(np.abs(X))
    assert np.max(np.abs(oracle.fft1d(X, inverse=True) - x)) < 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("ny,nx", [(10, 14), (50, 56), (6, 28)])
def test_fft2d_matches_direct_dft(ny, nx):
    rng = np.random.default_rng(nx * ny)
    x = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    ref = dft_matrix(ny, -1) @ x @ dft_matrix(nx, -1).T
    got = oracle.fft2d(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = oracle.fft2d(got, inverse=True)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("nx,ny,mt,my", [(56, 50, 3, 2), (28, 250, 5, -7), (112, 10, 13, 1)])
def test_single_mode_linear_propagation_is_exact(nx, ny, mt, my):
    # B = 0: a Fourier mode of Eq. 2a evolves as exp(lambda sigma) with
    # lambda = (1/4pi)(-ky^2)/(i kt) - A kt^2 (the regulariser is negligible)
    A, dt, n = 7e-4, 0.05, 30
    tau = -4.0 + 8.0 / nx * np.arange(nx)
    y = -8.0 + 16.0 / ny * np.arange(ny)
    kt, ky = 2 * np.pi * mt / 8.0, 2 * np.pi * my / 16.0
    phase = kt * tau[None, :] + ky * y[:, None]
    p = oracle.Params(nx=nx, ny=ny, dt=dt, B=0.0, A=A)
    u = oracle.run(p, np.cos(phase), n)
    lam = (1 / (4 * np.pi)) * (-ky ** 2) / (1j * kt) - A * kt ** 2
    assert np.max(np.abs(u - np.real(np.exp(lam * n * dt) * np.exp(1j * phase)))) < 1e-12


def test_mean_conserved_on_a_mixed_grid():
    w = inputs.config(1, nx=56, ny=50)
    p = oracle.Params(**inputs.oracle_params(w))
    u, hist = oracle.run(p, w.u0, 12, want_hist=True)
    m0 = np.mean(w.u0)
    assert np.all(np.abs(hist[:, 0] - m0) < 1e-15 + 1e-13 * abs(m0))
    row_means = u.mean(axis=1)
    assert np.max(np.abs(row_means - row_means.mean())) < 1e-12


def test_mixed_grid_agrees_with_the_same_field_on_a_finer_power_of_two_grid():
    """A smooth, band-limited initial field and B = 0: the scheme is exact for
    each mode, so the 7*8 x 50 grid and the 64 x 64 grid give the same field
    at their common points' positions (evaluated through the modes)."""
    A, dt, n = 2e-3, 0.1, 10
    modes = [(1, 0, 1.0), (2, 3, 0.5), (3, -2, 0.25)]

    def field(nx, ny, sig):
        tau = -4.0 + 8.0 / nx * np.arange(nx)
        y = -8.0 + 16.0 / ny * np.arange(ny)
        out = np.zeros((ny, nx))
        for mt, my, a in modes:
            kt, ky = 2 * np.pi * mt / 8.0, 2 * np.pi * my / 16.0
            lam = (1 / (4 * np.pi)) * (-ky ** 2) / (1j * kt) - A * kt ** 2
            out += a * np.real(np.exp(lam * sig) * np.exp(1j * (kt * tau[None, :] + ky * y[:, None])))
        return out

    for nx, ny in ((56, 50), (64, 64)):
        p = oracle.Params(nx=nx, ny=ny, dt=dt, B=0.0, A=A)
        u = oracle.run(p, field(nx, ny, 0.0), n)
        assert np.max(np.abs(u - field(nx, ny, n * dt))) < 1e-12
