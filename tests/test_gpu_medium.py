"""Parity of the random-medium path (Algorithm 1; the U_par / U_perp terms of
Eq. 2a in the flux form after Eq. 7) with the FP64 oracle, through the C ABI."""
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


@pytest.mark.parametrize("ny", [16, 256, 2048])
def test_coefficients_match_oracle(ny):
    api = _api()
    w = inputs.medium_config(64, ny, 10)
    plan = api.Plan.from_workload(w)
    p = oracle.Params(**inputs.oracle_params(w))
    for sigma in (0.0, 1.3, 57.0):
        a, b, c, mx = plan.medium_eval(sigma)
        ra, rb, rc = oracle.medium(p, sigma)
        for got, ref in ((a, ra), (b, rb), (c, rc)):
            assert np.max(np.abs(got - ref)) < 1e-14 * max(1.0, np.max(np.abs(ref)) / 1e-2)
        assert mx == np.max(np.abs(b))


@pytest.mark.parametrize("nx,ny", [(64, 16), (512, 128), (2048, 64)])
def test_rhs_matches_oracle(nx, ny):
    api = _api()
    w = inputs.medium_config(nx, ny, 10)
    plan = api.Plan.from_workload(w)
    sigma = 3.7
    b = plan.rhs(_dev(w.u0), sigma=sigma).cpu().numpy()
    ref = oracle.rhs(oracle.Params(**inputs.oracle_params(w)), w.u0, sigma=sigma)
    assert rel_linf(b, ref) < 1e-12


def test_run_fp64_parity():
    api = _api()
    w = inputs.medium_config(512, 256, 40)
    plan = api.Plan.from_workload(w)
    u = _dev(w.u0)
    plan.advance(u, w.n_steps)
    p = oracle.Params(**inputs.oracle_params(w))
    ref = oracle.run(p, w.u0, w.n_steps, threads=True)
    homog = oracle.run(oracle.Params(**inputs.oracle_params(w, mode_klam=None, mode_theta=None, mode_phase=None,
                                                            mode_amp=None)), w.u0, w.n_steps, threads=True)
    assert rel_l2(homog, ref) > 1e-3              # the medium changes the answer
    assert rel_linf(u.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("nx,ny,steps", [(512, 256, 40), (64, 16, 10), (1536, 40, 10)])
def test_run_fp32_error(nx, ny, steps):
    # FP32 y-flux sweep on column pairs: whole and partial CTAs of 256 columns,
    # 32-row blocks with a short last one, fewer rows than one block
    api = _api()
    w = inputs.medium_config(nx, ny, steps)
    plan = api.Plan.from_workload(w, precision="fp32")
    u = _dev(w.u0, torch.float32)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_l2(u.double().cpu().numpy(), ref) < 1e-5


def test_batch_shares_the_medium():
    api = _api()
    w = inputs.medium_config(256, 64, 12)
    u0 = np.stack([w.u0, 0.7 * w.u0[::-1]])
    plan = api.Plan.from_workload(w, batch=2)
    u = _dev(u0)
    plan.advance(u, w.n_steps)
    p = oracle.Params(**inputs.oracle_params(w))
    for i in range(2):
        ref = oracle.run(p, np.ascontiguousarray(u0[i]), w.n_steps)
        assert rel_linf(u[i].cpu().numpy(), ref) < 1e-11


def test_removing_the_medium_restores_the_homogeneous_path():
    api = _api()
    w = inputs.medium_config(128, 32, 5)
    plan = api.Plan.from_workload(w)
    plan.set_medium(None)
    a = _dev(w.u0)
    plan.advance(a, 5)
    w.medium = None
    ref_plan = api.Plan.from_workload(w)
    b = _dev(w.u0)
    ref_plan.advance(b, 5)
    assert torch.equal(a, b)


@pytest.mark.parametrize("prec,tol,method", [("fp64", 1e-10, "exprk22"), ("fp32", 3e-3, "exprk22"),
                                             ("fp64", 1e-10, "expeuler")])
def test_adjoint_matches_oracle(prec, tol, method):
    api = _api()
    w = inputs.medium_config(128, 64, 8)
    plan = api.Plan.from_workload(w, precision=prec, method=method)
    p = oracle.Params(**inputs.oracle_params(w, method=1 if method == "expeuler" else 0))
    g_end = 2 * w.dtau * oracle.run(p, w.u0, w.n_steps)
    ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g0 = plan.adjoint(_dev(w.u0, dt), _dev(g_end, dt), w.n_steps, ckpt_every=3)
    assert rel_linf(g0.double().cpu().numpy(), ref) < tol


def test_adjoint_finite_differences():
    from fd_util import central_fd_torch, fd_bound
    api = _api()
    w = inputs.medium_config(64, 32, 6)
    plan = api.Plan.from_workload(w)
    u0 = _dev(w.u0)

    y = u0.clone()
    plan.advance(y, w.n_steps)
    g0 = plan.adjoint(u0, 2 * w.dtau * y, w.n_steps, ckpt_every=4)
    rng = np.random.default_rng(31)
    for _ in range(3):
        v = _dev(rng.standard_normal(w.u0.shape))
        v /= v.norm()
        ad, fd = central_fd_torch(plan, u0, v, 3e-4, w.n_steps, w.dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-6, fd, float(g0.norm()), g0.numel()), (ad, fd)
