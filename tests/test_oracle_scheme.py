"""Pins of the oracle's ExpRK22 step (Eq. 5 / Eq. 11 / Algorithm 2) against
closed forms of the PDE (Eq. 2a): exact linear propagation of a Fourier mode,
conservation of the mean, the inviscid N-wave decay law, second order in
sigma, and the adjoint against finite differences."""
import os

import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs


def _grid(nx, ny, Lt=8.0, Ly=16.0):
    tau = -Lt / 2 + Lt / nx * np.arange(nx)
    y = -Ly / 2 + Ly / ny * np.arange(ny)
    return tau, y


@pytest.mark.parametrize("mt,my,A", [(3, 2, 7e-6), (1, 5, 3.4e-4), (7, 0, 1e-3), (2, -3, 0.0)])
def test_single_mode_linear_propagation_is_exact(mt, my, A):
    # B = 0: b == 0 and each Fourier mode exp(i(kt tau + ky y)) of Eq. 2a evolves
    # as exp(lambda sigma), lambda = (1/4pi) (-ky^2)/(i kt) - A kt^2
    nx, ny, dt, n = 32, 16, 0.05, 40
    tau, y = _grid(nx, ny)
    kt, ky = 2 * np.pi * mt / 8.0, 2 * np.pi * my / 16.0
    phase = kt * tau[None, :] + ky * y[:, None]
    u0 = np.cos(phase)
    p = oracle.Params(nx=nx, ny=ny, dt=dt, B=0.0, A=A)
    u = oracle.run(p, u0, n)
    lam = (1 / (4 * np.pi)) * (-ky ** 2) / (1j * kt) - A * kt ** 2
    exact = np.real(np.exp(lam * n * dt) * np.exp(1j * phase))
    assert np.max(np.abs(u - exact)) < 1e-12


def test_absorption_profile_term_closed_form():
    # with B = 0 and A(sigma) = A p(sigma), b(sigma, u) = (A(sigma) - A) d_tau^2 u
    nx, ny = 64, 4
    tau, _ = _grid(nx, ny)
    kt = 2 * np.pi * 5 / 8.0
    u = np.tile(np.sin(kt * tau), (ny, 1))
    prof = (1.0, 0.3, -0.02, 0.001)
    p = oracle.Params(nx=nx, ny=ny, dt=0.1, B=0.0, A=1e-3, A_prof=prof, has_profile=True)
    s = 2.5
    As = 1e-3 * (prof[0] + prof[1] * s + prof[2] * s * s + prof[3] * s ** 3)
    b = oracle.rhs(p, u, sigma=s)
    assert np.max(np.abs(b - (As - 1e-3) * (-kt * kt) * u)) < 1e-13


def test_mean_conserved_and_ymeans_annihilated():
    w = inputs.config(1, nx=64, ny=32)
    p = oracle.Params(**inputs.oracle_params(w))
    u, hist = oracle.run(p, w.u0, 20, want_hist=True)
    m0 = np.mean(w.u0)
    assert np.all(np.abs(hist[:, 0] - m0) < 1e-15 + 1e-13 * abs(m0))
    # the regularised multiplier removes every per-y tau-mean with k_y != 0
    row_means = u.mean(axis=1)
    assert np.max(np.abs(row_means - row_means.mean())) < 1e-12


def test_inviscid_nwave_amplitude_decay():
    # A = 0, y-uniform, no noise: diffraction is inert and Eq. 2a is Burgers'
    # equation; the N-wave peak decays as a0 (1 + sigma/sigma0)^(-1/2),
    # sigma0 = L / (B a0) (equal-area shock fitting)
    nx, ny, L, a0, B = 2048, 2, 1.0, 1.0, 0.05
    u0 = inputs.nwave(nx, ny, L=L, a0=a0, noise=0.0, y_gauss=False)
    dt = 0.4 * (8.0 / nx) / (B * a0)
    p = oracle.Params(nx=nx, ny=ny, dt=dt, B=B, A=0.0, lf_umax=1.1 * a0)
    sigma0 = L / (B * a0)
    u = u0
    done = 0
    for sig in (0.5 * sigma0, 1.5 * sigma0):
        n = int(round(sig / dt)) - done
        u = oracle.run(p, u, n, sigma0=done * dt)
        done += n
        a_exact = a0 / np.sqrt(1 + done * dt / sigma0)
        assert abs(u.max() - a_exact) < 0.01 * a_exact, (u.max(), a_exact)
        assert abs(-u.min() - a_exact) < 0.01 * a_exact


def test_second_order_in_sigma():
    # step halving against a reference 16x finer in sigma (cf. Table tab1)
    w = inputs.config(1, nx=128, ny=32)
    u0 = inputs.nwave(128, 32, noise=0.0)
    sig_end = 2.0
    base = dict(inputs.oracle_params(w))

    def solve(n):
        p = oracle.Params(**{**base, "dt": sig_end / n})
        return oracle.run(p, u0, n)

    tab = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "paper_tab1_convergence.txt"))
    lo, hi = np.nanmin(tab[:, 2]) - 0.25, np.nanmax(tab[:, 2]) + 0.25     # 1.90 .. 2.72
    ref = solve(320)
    errs = [np.linalg.norm(solve(n) - ref) / np.linalg.norm(ref) for n in (10, 20, 40)]
    betas = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(lo <= b <= hi for b in betas), (errs, betas)


def test_adjoint_matches_finite_differences():
    from fd_util import central_fd_numpy, fd_bound
    w = inputs.config(2, nx=32, ny=16, n_steps=6)
    p = oracle.Params(**inputs.oracle_params(w))
    n = 6
    dtau = w.dtau
    u_end = oracle.run(p, w.u0, n)
    g0 = oracle.adjoint(p, w.u0, 2 * dtau * u_end, n)
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(w.u0.shape)
        v /= np.linalg.norm(v)
        # h = 3e-6: O(h^2) truncation and the rounding of the factorised loss
        # difference both stay far below 1e-7 of the directional derivative
        ad, fd = central_fd_numpy(lambda x: oracle.run(p, x, n), w.u0, v, 3e-6, dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-7, fd, np.linalg.norm(g0), g0.size), (ad, fd)
