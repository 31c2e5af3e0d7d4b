"""Pins of the oracle's exponential Euler scheme (Sec. 3.2: the first stage of
Eq. 5 taken as the step).  It is exact for the linear part (a single Fourier
mode with B = 0 follows exp(lambda sigma)), first order in sigma as the paper
states, its one step is the first stage of ExpRK22, and its transpose agrees
with central finite differences."""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs


def test_single_mode_linear_propagation_is_exact():
    nx, ny, dt, n = 32, 16, 0.37, 9
    p = oracle.Params(nx=nx, ny=ny, dt=dt, B=0.0, A=7e-4, method=1)
    tau = -4.0 + 8.0 * np.arange(nx) / nx
    y = -8.0 + 16.0 * np.arange(ny) / ny
    mt, my = 3, 2
    kt, ky = 2 * np.pi * mt / 8.0, 2 * np.pi * my / 16.0
    u0 = np.cos(kt * tau)[None, :] * np.cos(ky * y)[:, None]
    # Eq. 2a for this mode: d/dsigma of exp(i kt tau) cos(ky y) is
    # lambda = -(1/4pi) ky^2 / (i kt) - A kt^2 (regulariser negligible here)
    lam = -(1.0 / (4 * np.pi)) * ky * ky / (1j * kt) - 7e-4 * kt * kt
    ref = np.real(np.exp(lam * n * dt) * np.exp(1j * kt * tau))[None, :] * np.cos(ky * y)[:, None]
    got = oracle.run(p, u0, n)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_first_order_in_sigma():
    w = inputs.config(1, nx=128, ny=32)
    u0 = inputs.nwave(128, 32, noise=0.0)
    sig_end = 2.0
    base = dict(inputs.oracle_params(w))

    def solve(n, method):
        return oracle.run(oracle.Params(**{**base, "dt": sig_end / n, "method": method}), u0, n)

    ref = solve(640, 0)                      # ExpRK22, far finer in sigma
    errs = [np.linalg.norm(solve(n, 1) - ref) / np.linalg.norm(ref) for n in (20, 40, 80)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 <= r <= 1.2 for r in rates), (errs, rates)


def test_one_step_is_the_first_exprk22_stage():
    w = inputs.config(2, nx=64, ny=16, n_steps=1)
    p22 = oracle.Params(**inputs.oracle_params(w))
    pe = oracle.Params(**inputs.oracle_params(w, method=1))
    _, ustar = oracle.run(p22, w.u0, 1, want_ustar=True)
    assert np.array_equal(oracle.run(pe, w.u0, 1), ustar)


def test_adjoint_matches_finite_differences():
    from fd_util import central_fd_numpy, fd_bound
    w = inputs.config(2, nx=32, ny=16, n_steps=6)
    p = oracle.Params(**inputs.oracle_params(w, method=1))
    n = 6
    dtau = w.dtau
    g0 = oracle.adjoint(p, w.u0, 2 * dtau * oracle.run(p, w.u0, n), n)
    rng = np.random.default_rng(12)
    for _ in range(3):
        v = rng.standard_normal(w.u0.shape)
        v /= np.linalg.norm(v)
        ad, fd = central_fd_numpy(lambda x: oracle.run(p, x, n), w.u0, v, 3e-6, dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-7, fd, np.linalg.norm(g0), g0.size), (ad, fd)
