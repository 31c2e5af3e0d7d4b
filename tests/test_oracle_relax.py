"""Pins of the oracle's relaxation term (an extra diagonal term of the linear
operator of Eq. 2a / Eq. 11, added to the multiplier z).

A relaxation process of strength C and relaxation time theta contributes
C d_tau^2 q, where q solves theta dq/dtau + q = V and decays into the past,
i.e. q is the causal exponential average of V:
    q(tau) = (1/theta) int_0^inf exp(-s/theta) V(tau - s) ds.
These tests evaluate that average for a Fourier mode by numerical quadrature
(scipy's QAWF routine), independently of the closed form the oracle uses, and
check the oracle's propagator E = exp(dsigma L) against it; the limit of a
vanishing relaxation time must reduce to plain absorption A + C.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle


def relax_symbol_quad(k, C, theta):
    """C (i k)^2 (1/theta) int_0^inf exp(-s/theta) exp(-i k s) ds, by quadrature."""
    f = lambda s: np.exp(-s / theta) / theta
    ic, _ = integrate.quad(f, 0.0, np.inf, weight="cos", wvar=k)
    is_, _ = integrate.quad(f, 0.0, np.inf, weight="sin", wvar=k)
    return C * (-(k * k)) * (ic - 1j * is_)


@pytest.mark.parametrize("C,theta", [(1e-3, 0.05), (4e-4, 0.4), (2e-3, 0.01)])
def test_propagator_matches_quadrature(C, theta):
    nx, ny, dt, A = 64, 4, 0.2, 7e-6
    p = oracle.Params(nx=nx, ny=ny, dt=dt, A=A, relax_C=(C,), relax_theta=(theta,))
    E, _, _ = oracle.tables(p)
    L = p.tau_max - p.tau_min
    for m in (1, 3, 7, 15, 31):
        k = 2 * np.pi * m / L
        ref = np.exp(dt * (-A * k * k + relax_symbol_quad(k, C, theta)))
        assert abs(E[0, m] - ref) < 1e-12 * abs(ref), (m, E[0, m], ref)
        # the mirrored frequency carries the conjugate (real fields stay real)
        assert abs(E[0, nx - m] - np.conj(ref)) < 1e-12 * abs(ref)


def test_two_processes_add_and_nyquist_is_real():
    nx, ny, dt, A = 32, 2, 0.3, 7e-6
    procs = ((1e-3, 0.05), (5e-4, 0.3))
    p = oracle.Params(nx=nx, ny=ny, dt=dt, A=A, relax_C=tuple(c for c, _ in procs),
                      relax_theta=tuple(t for _, t in procs))
    E, _, _ = oracle.tables(p)
    L = p.tau_max - p.tau_min
    for m in (2, 5, 11):
        k = 2 * np.pi * m / L
        ref = np.exp(dt * (-A * k * k + sum(relax_symbol_quad(k, c, t) for c, t in procs)))
        assert abs(E[0, m] - ref) < 1e-12 * abs(ref)
    # tau-Nyquist: the real (even) part of the multiplier only
    kN = np.pi * nx / L
    ref = np.exp(dt * (-A * kN * kN + sum(relax_symbol_quad(kN, c, t) for c, t in procs).real))
    assert E[0, nx // 2].imag == 0.0
    assert abs(E[0, nx // 2].real - ref) < 1e-12 * ref


def test_relaxation_is_dissipative():
    p = oracle.Params(nx=64, ny=8, dt=0.5, relax_C=(2e-3, 1e-3), relax_theta=(0.02, 0.5))
    E, _, _ = oracle.tables(p)
    assert np.all(np.abs(E) <= 1.0 + 1e-15)


def test_vanishing_relaxation_time_is_absorption():
    """theta -> 0: C d_tau^2 (1 + theta d_tau)^-1 -> C d_tau^2, extra absorption."""
    nx, ny, n = 128, 16, 20
    base = dict(nx=nx, ny=ny, dt=0.01, B=0.05, lf_umax=1.2)
    C = 3e-3
    pr = oracle.Params(A=7e-6, relax_C=(C,), relax_theta=(1e-13,), **base)
    pa = oracle.Params(A=7e-6 + C, **base)
    Er, _, _ = oracle.tables(pr)
    Ea, _, _ = oracle.tables(pa)
    assert np.max(np.abs(Er - Ea)) < 1e-11
    rng = np.random.default_rng(3)
    tau = np.linspace(-4, 4, nx, endpoint=False)
    u0 = np.outer(np.exp(-np.linspace(-8, 8, ny, endpoint=False) ** 2 / 16), np.sin(2 * np.pi * tau / 8))
    u0 = u0 + 1e-3 * rng.uniform(-1, 1, u0.shape)
    ur = oracle.run(pr, u0, n)
    ua = oracle.run(pa, u0, n)
    assert np.max(np.abs(ur - ua)) < 1e-10 * np.max(np.abs(ua))


def test_without_processes_nothing_changes():
    p0 = oracle.Params(nx=32, ny=8, dt=0.1)
    p1 = oracle.Params(nx=32, ny=8, dt=0.1, relax_C=(0.0,), relax_theta=(0.1,))
    for a, b in zip(oracle.tables(p0), oracle.tables(p1)):
        assert np.array_equal(a, b)
