"""Pins of the oracle's random-medium terms (Algorithm 1, Eq. 2a / Eq. 3 and
the flux form that follows Eq. 7).

The field: divergence-free (the mode vectors are orthogonal to their wave
vectors), its y-derivative against central differences of the field itself,
and its size against the bound the paper states for its parameters (0.05).
The right-hand side: without modes it is the homogeneous one bit for bit; a
constant U_par is advection along tau with speed 2 pi U_par and a constant
U_perp advection along y (b -> 2 pi U_par du/dtau, -U_perp du/dy, fifth order
on smooth data); with a y-dependent U_perp the flux form d_y(U_perp u) minus
the source d_y U_perp u converges to U_perp du/dy.
"""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs


def _params(nx, ny, med, **kw):
    return oracle.Params(nx=nx, ny=ny, dt=0.01, mode_klam=med.klam, mode_theta=med.theta, mode_phase=med.phase,
                         mode_amp=med.amp, **kw)


def _one_mode(klam, theta, phase, amp):
    return inputs.Medium(klam=np.array([klam]), theta=np.array([theta]), phase=np.array([phase]),
                         amp=np.array([amp]))


def test_field_is_divergence_free():
    med = inputs.random_medium(7, 64)
    p = _params(8, 64, med)
    for sigma in (0.0, 3.7, 25.0):
        h = 1e-4
        a_p, _, _ = oracle.medium(p, sigma + h)
        a_m, _, _ = oracle.medium(p, sigma - h)
        _, _, dperp = oracle.medium(p, sigma)
        div = (a_p - a_m) / (2 * h) + dperp
        assert np.max(np.abs(div)) < 1e-8 * max(1.0, np.max(np.abs(dperp)) / 1e-3)


def test_field_y_derivative_matches_differences():
    med = inputs.random_medium(8, 64)
    h = 1e-4
    base = dict(y_min=-8.0, y_max=8.0)
    p0 = _params(8, 32, med, **base)
    pp = _params(8, 32, med, y_min=-8.0 + h, y_max=8.0 + h)
    pm = _params(8, 32, med, y_min=-8.0 - h, y_max=8.0 - h)
    for sigma in (0.5, 11.0):
        _, up, _ = oracle.medium(pp, sigma)
        _, um, _ = oracle.medium(pm, sigma)
        _, _, d = oracle.medium(p0, sigma)
        assert np.max(np.abs((up - um) / (2 * h) - d)) < 1e-8


def test_field_within_the_papers_bound():
    """The paper states |U_par|, |U_perp| <= 0.05 for its parameters (Sec. 2)."""
    med = inputs.random_medium(11, 128)
    p = _params(8, 256, med)
    mx_par = mx_perp = 0.0
    for sigma in np.linspace(0.0, 200.0, 81):
        a, b, _ = oracle.medium(p, sigma)
        mx_par, mx_perp = max(mx_par, np.max(np.abs(a))), max(mx_perp, np.max(np.abs(b)))
    assert 1e-3 < mx_par <= 0.05 and 1e-3 < mx_perp <= 0.05


def test_without_modes_rhs_is_homogeneous():
    w = inputs.config(1, nx=64, ny=16)
    p0 = oracle.Params(**inputs.oracle_params(w))
    zero = inputs.Medium(klam=np.array([0.3, 1.0]), theta=np.array([0.2, 2.0]), phase=np.array([0.1, 0.5]),
                         amp=np.zeros(2))
    pz = oracle.Params(**inputs.oracle_params(w, mode_klam=zero.klam, mode_theta=zero.theta,
                                              mode_phase=zero.phase, mode_amp=zero.amp))
    assert np.array_equal(oracle.weno_rhs(p0, w.u0, 0.3), oracle.weno_rhs(pz, w.u0, 0.3))
    assert np.array_equal(oracle.run(p0, w.u0, 3), oracle.run(pz, w.u0, 3))


def _order(errs, ns):
    return np.polyfit(np.log(ns), np.log(errs), 1)[0] * -1


def test_constant_upar_is_tau_advection():
    amp = 0.04
    med = _one_mode(0.0, 1.5 * np.pi, 0.0, amp)       # U_par = amp, U_perp ~ 0, both constant
    errs, ns = [], [64, 128, 256, 512]
    for nx in ns:
        p = _params(nx, 4, med, B=0.0, lf_umax=1.0)
        tau = -4.0 + 8.0 * np.arange(nx) / nx
        u = np.tile(np.sin(2 * np.pi * tau / 8) + 0.3 * np.cos(6 * np.pi * tau / 8), (4, 1))
        exact = 2 * np.pi * amp * (2 * np.pi / 8) * np.tile(
            np.cos(2 * np.pi * tau / 8) - 0.9 * np.sin(6 * np.pi * tau / 8), (4, 1))
        errs.append(np.mean(np.abs(oracle.weno_rhs(p, u, 0.0) - exact)))
    assert errs[-1] < 1e-9
    assert _order(errs, ns) > 4.5


def test_constant_uperp_is_y_advection():
    amp = 0.03
    med = _one_mode(0.0, 0.0, 0.0, amp)               # U_perp = amp, U_par = 0
    errs, ns = [], [64, 128, 256, 512]
    for ny in ns:
        p = _params(8, ny, med, B=0.0, lf_umax=1.0)
        y = -8.0 + 16.0 * np.arange(ny) / ny
        u = np.tile((np.sin(2 * np.pi * y / 16) + 0.5 * np.cos(4 * np.pi * y / 16))[:, None], (1, 8))
        exact = -amp * (2 * np.pi / 16) * np.tile(
            (np.cos(2 * np.pi * y / 16) - np.sin(4 * np.pi * y / 16))[:, None], (1, 8))
        errs.append(np.mean(np.abs(oracle.weno_rhs(p, u, 0.0) - exact)))
    assert errs[-1] < 1e-9
    assert _order(errs, ns) > 4.5


def test_flux_form_with_variable_uperp():
    """-d_y(U_perp u) + (d_y U_perp) u -> -U_perp du/dy for smooth u (tau-uniform,
    vanishing towards the periodic y-boundary)."""
    med = _one_mode(0.7, 0.25 * np.pi, 0.4, 0.03)
    errs, ns = [], [128, 256, 512, 1024]
    for ny in ns:
        p = _params(8, ny, med, B=0.0, lf_umax=1.0)
        y = -8.0 + 16.0 * np.arange(ny) / ny
        g = np.exp(-y ** 2 / 2) * (1 + 0.3 * y)
        dg = np.exp(-y ** 2 / 2) * (0.3 - y * (1 + 0.3 * y))
        _, uperp, _ = oracle.medium(p, 0.0)
        exact = np.tile((-uperp * dg)[:, None], (1, 8))
        errs.append(np.max(np.abs(oracle.weno_rhs(p, np.tile(g[:, None], (1, 8)), 0.0) - exact)))
    assert errs[-1] < 1e-8
    assert _order(errs, ns) > 4.0


def test_transpose_is_adjoint_of_linearisation():
    """<J^T mu, v> = <mu, J v> with J v from central differences of the
    medium's b (the transposed tau- and y-fluxes and the source)."""
    w = inputs.medium_config(64, 32, 4)
    p = oracle.Params(**inputs.oracle_params(w))
    rng = np.random.default_rng(21)
    u = w.u0
    sigma = 5.3
    for _ in range(3):
        mu = rng.standard_normal(u.shape)
        v = rng.standard_normal(u.shape)
        h = 1e-6
        jv = (oracle.weno_rhs(p, u + h * v, sigma) - oracle.weno_rhs(p, u - h * v, sigma)) / (2 * h)
        jtmu = oracle.weno_rhs_T(p, u, mu, sigma)
        lhs, rhs = np.sum(jtmu * v), np.sum(mu * jv)
        assert abs(lhs - rhs) < 1e-7 * (np.linalg.norm(jtmu) * np.linalg.norm(v)), (lhs, rhs)


def test_adjoint_matches_finite_differences():
    from fd_util import central_fd_numpy, fd_bound
    w = inputs.medium_config(32, 16, 5)
    p = oracle.Params(**inputs.oracle_params(w))
    n, dtau = 5, w.dtau
    g0 = oracle.adjoint(p, w.u0, 2 * dtau * oracle.run(p, w.u0, n), n)
    rng = np.random.default_rng(22)
    for _ in range(3):
        v = rng.standard_normal(w.u0.shape)
        v /= np.linalg.norm(v)
        ad, fd = central_fd_numpy(lambda x: oracle.run(p, x, n), w.u0, v, 3e-6, dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-7, fd, np.linalg.norm(g0), g0.size), (ad, fd)
