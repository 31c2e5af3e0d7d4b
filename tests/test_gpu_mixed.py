"""Parity of the mixed-radix path (grids whose sizes are not powers of two,
such as the 7 * 2^k x 1250 * 2^k grids of Table 1) with the FP64 oracle,
through the C ABI.

The same bars as the power-of-two path: FP64 relative L-infinity within 1e-11
after whole runs (tighter for single operations), FP32 relative l2 within
1e-5.  Sizes include single and several column tiles, odd half lengths
(nx / 2 odd), every radix (2, 3, 4, 5, 7, 8), the random medium, exponential
Euler, batches and the adjoint (against the oracle's transposed step and
finite differences); the paper's largest grid (3584 x 10000) is checked
against the closed form of a propagating Fourier mode, which holds at any
size.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _api():
    from paper_2103_06080_b300 import api
    return api


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("nx,ny", [(14, 6), (56, 50), (448, 10), (30, 18), (3584, 4), (210, 42)])
def test_tau_fft_matches_dft(nx, ny):
    api = _api()
    rng = np.random.default_rng(nx + ny)
    u = rng.standard_normal((ny, nx))
    plan = api.Plan(nx=nx, ny=ny, dt=0.01)
    V = plan.tau_fft(_dev(u), -1).cpu().numpy()
    ref = np.stack([oracle.fft1d(u[j]) for j in range(ny)]) / nx
    got = V[..., 0] + 1j * V[..., 1]
    assert np.max(np.abs(got[:, 1:] - ref[:, 1:nx // 2])) < 1e-14 * np.max(np.abs(ref)) + 1e-15
    assert np.max(np.abs(got[:, 0].real - ref[:, 0].real)) < 1e-14
    assert np.max(np.abs(got[:, 0].imag - ref[:, nx // 2].real)) < 1e-14
    back = plan.tau_fft(torch.tensor(V, device="cuda"), +1).cpu().numpy()
    assert np.max(np.abs(back - u)) < 1e-13 * np.max(np.abs(u))


@pytest.mark.parametrize("nx,ny", [(56, 50), (448, 250), (30, 42)])
def test_rhs_matches_oracle(nx, ny):
    api = _api()
    w = inputs.config(2, nx=nx, ny=ny, n_steps=10)
    plan = api.Plan.from_workload(w)
    b = plan.rhs(_dev(w.u0), sigma=0.7).cpu().numpy()
    ref = oracle.rhs(oracle.Params(**inputs.oracle_params(w)), w.u0, sigma=0.7)
    assert rel_linf(b, ref) < 1e-12


@pytest.mark.parametrize("nx,ny,steps", [(56, 50, 40), (448, 250, 30), (210, 1250, 6), (14, 6, 20)])
def test_run_fp64_parity(nx, ny, steps):
    api = _api()
    w = inputs.config(2, nx=nx, ny=ny, n_steps=steps)
    plan = api.Plan.from_workload(w)
    u = _dev(w.u0)
    st, d = plan.advance(u, w.n_steps, diag=True)
    assert st == 0
    p = oracle.Params(**inputs.oracle_params(w))
    ref, hist = oracle.run(p, w.u0, w.n_steps, threads=True, want_hist=True)
    assert rel_linf(u.cpu().numpy(), ref) < 1e-11
    gh = plan.diag_history(w.n_steps)[:, 0, :]
    assert np.allclose(gh[1:, 1], hist[:-1, 1], rtol=1e-11)
    assert abs(d[0]["energy"] - hist[-1, 1]) < 1e-11 * hist[-1, 1]
    assert np.max(np.abs(gh[:, 0] - gh[0, 0])) < 1e-14


# Columns of 10000 points (the column length of Set 4, Table 1) with the
# nonlinear term: FP32 runs them as tiles of two columns at one CTA per SM
# (the compensated state's transforms on plain FP32 twiddles), FP64 as single
# columns; both against the oracle.  The y extent grows with ny so that dy is
# that of the 4096 x 2048 grid: on [-8, 8] the diffraction phase
# dsigma ky^2 / (4 pi k_tau) of the highest ky would reach 1e5-1e6 rad, where
# one rounding of the phase in either side's FP64 tables is already ~1e-10.
@pytest.mark.parametrize("prec,nx,steps", [("fp32", 56, 20), ("fp64", 56, 10)])
def test_run_long_columns(prec, nx, steps):
    api = _api()
    w = inputs.config(2, nx=nx, ny=10000, n_steps=steps)
    w = dataclasses.replace(w, y_min=-8.0 * 10000 / 2048, y_max=8.0 * 10000 / 2048)
    plan = api.Plan.from_workload(w, precision=prec)
    u = _dev(w.u0, torch.float64 if prec == "fp64" else torch.float32)
    st, _ = plan.advance(u, w.n_steps, diag=True)
    assert st == 0
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    got = u.double().cpu().numpy()
    if prec == "fp64":
        assert rel_linf(got, ref) < 1e-11
    else:
        assert rel_l2(got, ref) < 1e-5
        assert rel_linf(got, ref) < 1e-4


def test_one_step_stages_match_oracle():
    api = _api()
    w = inputs.config(2, nx=448, ny=50, n_steps=5)
    plan = api.Plan.from_workload(w)
    s0 = 2 * w.dt
    us, un = plan.step_stages(_dev(w.u0), sigma0=s0)
    ref_un, ref_us = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 1, sigma0=s0, want_ustar=True)
    assert rel_linf(us.cpu().numpy(), ref_us) < 1e-13
    assert rel_linf(un.cpu().numpy(), ref_un) < 1e-13


def test_fp32_error_against_fp64_oracle():
    api = _api()
    w = inputs.config(3, nx=448, ny=250, n_steps=100)
    plan = api.Plan.from_workload(w, precision="fp32")
    u = _dev(w.u0, torch.float32)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    got = u.double().cpu().numpy()
    assert rel_l2(got, ref) < 1e-5
    assert rel_linf(got, ref) < 1e-4


# 448 x 250 (12 steps), and the exact grids of Sets 1 and 2 of Table 1 (448 x
# 1250, 896 x 2500; a few steps) that bench.py times: their column tiles are
# narrowed to leave tiles for most SMs and their y sweeps take 16-32 rows per
# CTA, so these are the launch shapes of the paper-grid measurement
@pytest.mark.parametrize("prec,tol,nx,ny,steps", [("fp64", 1e-11, 448, 250, 12), ("fp32", 1e-5, 448, 250, 12),
                                                  ("fp64", 1e-11, 448, 1250, 4), ("fp32", 1e-5, 448, 1250, 4),
                                                  ("fp64", 1e-11, 896, 2500, 3), ("fp32", 1e-5, 896, 2500, 3)])
def test_random_medium_run(prec, tol, nx, ny, steps):
    api = _api()
    w = inputs.medium_config(nx, ny, steps)
    plan = api.Plan.from_workload(w, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = _dev(w.u0, dt)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    got = u.double().cpu().numpy()
    assert (rel_linf if prec == "fp64" else rel_l2)(got, ref) < tol


def test_expeuler_and_relaxation_run():
    api = _api()
    w = inputs.config(2, nx=56, ny=50, n_steps=15)
    kw = dict(relax_C=(1e-3,), relax_theta=(0.05,))
    plan = api.Plan.from_workload(w, method="expeuler", **kw)
    u = _dev(w.u0)
    plan.advance(u, w.n_steps)
    p = oracle.Params(**inputs.oracle_params(w, method=1, relax_C=(1e-3,), relax_theta=(0.05,)))
    assert rel_linf(u.cpu().numpy(), oracle.run(p, w.u0, w.n_steps)) < 1e-11


def test_batch_instances_are_independent():
    api = _api()
    w = inputs.config(2, nx=112, ny=250, n_steps=8)
    u0 = np.stack([w.u0, -0.5 * w.u0[::-1]])
    plan = api.Plan.from_workload(w, batch=2)
    u = _dev(u0)
    plan.advance(u, w.n_steps)
    p = oracle.Params(**inputs.oracle_params(w))
    for i in range(2):
        assert rel_linf(u[i].cpu().numpy(), oracle.run(p, np.ascontiguousarray(u0[i]), w.n_steps)) < 1e-11


def test_mixed_kernels_on_a_power_of_two_grid():
    """transforms="mixed" runs the mixed-radix kernels on a power-of-two grid:
    the result agrees with the radix-8/16 kernels and with the oracle."""
    api = _api()
    w = inputs.config(2, nx=512, ny=128, n_steps=30)
    a = _dev(w.u0)
    api.Plan.from_workload(w).advance(a, w.n_steps)
    b = _dev(w.u0)
    pm = api.Plan.from_workload(w, transforms="mixed")
    assert pm.info()["transforms"] == "mixed"
    pm.advance(b, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_linf(b.cpu().numpy(), ref) < 1e-11
    assert rel_linf(b.cpu().numpy(), a.cpu().numpy()) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_paper_grid_single_mode_closed_form(prec, tol):
    """Set 4 of Table 1 (N_theta = 7 * 512 = 3584, N_rho = 10000), B = 0: a
    Fourier mode follows exp(lambda sigma) exactly (Eq. 2a), so every point of
    the full grid is checked against the closed form."""
    api = _api()
    nx, ny, dt, n = 3584, 10000, 0.05, 6
    A = 7e-4
    mt, my = 5, 3
    kt, ky = 2 * np.pi * mt / 8.0, 2 * np.pi * my / 16.0
    plan = api.Plan(nx=nx, ny=ny, dt=dt, precision=prec, B=1e-300, A=A, lf_umax=1.0)
    tau = torch.arange(nx, dtype=torch.float64, device="cuda") * (8.0 / nx) - 4.0
    y = torch.arange(ny, dtype=torch.float64, device="cuda") * (16.0 / ny) - 8.0
    phase = kt * tau[None, :] + ky * y[:, None]
    dtype = torch.float64 if prec == "fp64" else torch.float32
    u = torch.cos(phase).to(dtype).contiguous()
    plan.advance(u, n)
    lam = (1 / (4 * np.pi)) * (-ky ** 2) / (1j * kt) - A * kt ** 2
    z = np.exp(lam * n * dt)
    exact = z.real * torch.cos(phase) - z.imag * torch.sin(phase)
    err = float((u.double() - exact).abs().max())
    assert err < tol


def test_unsupported_sizes_and_features_are_refused():
    api = _api()
    for nx, ny in ((22, 16), (15, 10), (64, 26), (56, 13)):   # prime factor 11 or 13, odd sizes
        with pytest.raises(Exception):
            api.Plan(nx=nx, ny=ny, dt=0.01)
    w = inputs.config(2, nx=56, ny=50, n_steps=4)
    with pytest.raises(Exception):
        api.BatchedPlan([w], precision="fp64", mode="persistent")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_streams_with_mixed_and_power_of_two_instances(prec):
    """One graph launch advancing instances of the paper's grid shapes next to
    power-of-two ones: every instance equals its own plan, bit for bit."""
    api = _api()
    ws = [inputs.config(2, nx=448, ny=250, n_steps=6), inputs.config(2, nx=512, ny=128, n_steps=6),
          inputs.config(2, nx=56, ny=50, n_steps=6)]
    for w in ws:
        w.precision = prec
    dt = torch.float64 if prec == "fp64" else torch.float32
    bp = api.BatchedPlan(ws, precision=prec, mode="streams", autotune=False)
    us = [_dev(w.u0, dt) for w in ws]
    st, _ = bp.advance(us, 6, diag=True)
    assert st == 0
    for w, u in zip(ws, us):
        p = api.Plan.from_workload(w, precision=prec)
        v = _dev(w.u0, dt)
        p.advance(v, 6)
        assert torch.equal(u, v), (w.nx, w.ny)
        p.close()
    bp.close()


@pytest.mark.parametrize("nx,ny,prec,tol,method,medium", [
    (56, 50, "fp64", 1e-10, "exprk22", False), (448, 250, "fp64", 1e-10, "exprk22", False),
    (30, 18, "fp64", 1e-10, "expeuler", False), (112, 50, "fp64", 1e-10, "exprk22", True),
    (448, 250, "fp32", 3e-3, "exprk22", False)])
def test_adjoint_matches_oracle(nx, ny, prec, tol, method, medium):
    api = _api()
    n = 8
    w = inputs.medium_config(nx, ny, n) if medium else inputs.config(2, nx=nx, ny=ny, n_steps=n)
    plan = api.Plan.from_workload(w, precision=prec, method=method)
    p = oracle.Params(**inputs.oracle_params(w, method=1 if method == "expeuler" else 0))
    g_end = 2 * w.dtau * oracle.run(p, w.u0, n)
    ref = oracle.adjoint(p, w.u0, g_end, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g0 = plan.adjoint(_dev(w.u0, dt), _dev(g_end, dt), n, ckpt_every=3)
    assert rel_linf(g0.double().cpu().numpy(), ref) < tol


def test_adjoint_finite_differences_on_a_paper_grid_shape():
    from fd_util import central_fd_torch, fd_bound
    # Set 1 of Table 1 (448 x 1250), a few steps: <g0, v> against central
    # differences with h = 3e-4 (fd_util: h where truncation and rounding of
    # the difference balance; with h = 1e-6 its rounding alone is ~4e-5)
    api = _api()
    w = inputs.config(2, nx=448, ny=1250, n_steps=4)
    plan = api.Plan.from_workload(w)
    u0 = _dev(w.u0)

    y = u0.clone()
    plan.advance(y, w.n_steps)
    g0 = plan.adjoint(u0, 2 * w.dtau * y, w.n_steps, ckpt_every=2)
    rng = np.random.default_rng(41)
    for _ in range(2):
        v = _dev(rng.standard_normal(w.u0.shape))
        v /= v.norm()
        ad, fd = central_fd_torch(plan, u0, v, 3e-4, w.n_steps, w.dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-6, fd, float(g0.norm()), g0.numel()), (ad, fd)
