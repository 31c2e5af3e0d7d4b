"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64: element-wise relative L-infinity (max|gpu - oracle| / max|oracle|)
within 1e-11 after whole runs, tighter for single operations.  FP32: relative
l2 within 1e-5 (error of FP32 bulk arithmetic with FP64 tables, against the
FP64 oracle).  Sizes span several column tiles and row blocks; edge cases
cover the smallest and largest supported grids and batches.
"""
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


@pytest.mark.parametrize("nx,ny", [(8, 2), (64, 8), (512, 4), (8192, 2)])
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tables_match_oracle(prec):
    api = _api()
    w = inputs.config(1, nx=64, ny=32)
    plan = api.Plan.from_workload(w, precision=prec)
    E, P1, P2 = plan.tables()
    p = oracle.Params(**inputs.oracle_params(w))
    oE, oP1, oP2 = oracle.tables(p)
    nl, nm = w.ny // 2 + 1, w.nx // 2 + 1
    tol = 1e-13 if prec == "fp64" else 2e-7
    for got, ref in ((E, oE), (P1, oP1), (P2, oP2)):
        ref = ref[:nl, :nm]
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        assert np.max(err[np.abs(ref) > 1e-280]) < tol


@pytest.mark.parametrize("nx,ny,profile", [(64, 8, False), (512, 64, True), (2048, 4, True)])
def test_rhs_matches_oracle(nx, ny, profile):
    api = _api()
    w = inputs.config(2 if profile else 1, nx=nx, ny=ny, n_steps=50)
    plan = api.Plan.from_workload(w, precision="fp64")
    sigma = 0.37 * w.n_steps * w.dt
    b = plan.rhs(_dev(w.u0), sigma=sigma).cpu().numpy()
    ref = oracle.rhs(oracle.Params(**inputs.oracle_params(w)), w.u0, sigma=sigma)
    assert rel_linf(b, ref) < 1e-12


def test_one_step_stages_match_oracle():
    api = _api()
    w = inputs.config(2, nx=256, ny=64, n_steps=20)
    plan = api.Plan.from_workload(w, precision="fp64")
    s0 = 3 * w.dt
    us, un = plan.step_stages(_dev(w.u0), sigma0=s0)
    p = oracle.Params(**inputs.oracle_params(w))
    ref_un, ref_us = oracle.run(p, w.u0, 1, sigma0=s0, want_ustar=True)
    assert rel_linf(us.cpu().numpy(), ref_us) < 1e-13
    assert rel_linf(un.cpu().numpy(), ref_un) < 1e-13


def test_config1_full_run_fp64_parity():
    # the full plain-method workload: 512 x 256, 200 steps, relative L-inf <= 1e-11
    api = _api()
    w = inputs.config(1)
    plan = api.Plan.from_workload(w, precision="fp64")
    u = _dev(w.u0)
    st, d = plan.advance(u, w.n_steps, diag=True)
    assert st == 0
    p = oracle.Params(**inputs.oracle_params(w))
    ref, hist = oracle.run(p, w.u0, w.n_steps, threads=True, want_hist=True)
    assert rel_linf(u.cpu().numpy(), ref) < 1e-11
    # diagnostics (FP64): state at the start of every step, and the final state
    gh = plan.diag_history(w.n_steps)[:, 0, :]
    od = oracle.diag(p, w.u0)
    assert abs(gh[0, 0] - od[0]) < 1e-15 and abs(gh[0, 1] - od[1]) < 1e-12 * od[1]
    assert np.allclose(gh[1:, 1], hist[:-1, 1], rtol=1e-11)
    assert np.allclose(gh[1:, 2], hist[:-1, 2], rtol=1e-11)
    assert abs(d[0]["energy"] - hist[-1, 1]) < 1e-11 * hist[-1, 1]
    # mean conserved to roundoff over the run
    assert np.max(np.abs(gh[:, 0] - gh[0, 0])) < 1e-14


def test_stratified_run_fp64_parity():
    api = _api()
    w = inputs.config(2, nx=512, ny=128, n_steps=60)
    plan = api.Plan.from_workload(w, precision="fp64")
    u = _dev(w.u0)
    plan.advance(u, w.n_steps, sigma0=0.0)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_linf(u.cpu().numpy(), ref) < 1e-11


def test_fp32_error_against_fp64_oracle():
    api = _api()
    w = inputs.config(3, nx=512, ny=256, n_steps=100)
    plan = api.Plan.from_workload(w, precision="fp32")
    u = _dev(w.u0, torch.float32)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    got = u.double().cpu().numpy()
    assert rel_l2(got, ref) < 1e-5
    assert rel_linf(got, ref) < 1e-4


# Column kernels chosen through the plan options: the TMA-staged Stockham
# tiles (FP32 plans the column-pair kernels do not take; FP64 on request) and
# the per-tile kernels with plain loads (FP64's default, and every plan the
# staged ones do not fit: ny = 4096 in FP32 needs 1024 threads per tile).
@pytest.mark.parametrize("prec,col,nx,ny,batch,steps", [
    ("fp32", "tma", 1024, 512, 1, 30),
    ("fp32", "tile", 1024, 512, 1, 30),
    ("fp32", "tma", 256, 16, 2, 20),
    ("fp32", "tile", 64, 4096, 1, 6),
    ("fp64", "tma", 512, 128, 2, 20),
    ("fp64", "tma", 32, 16, 1, 20),
])
def test_column_kernel_variants(prec, col, nx, ny, batch, steps):
    api = _api()
    w = inputs.config(2, nx=nx, ny=ny, n_steps=steps)
    u0 = np.stack([w.u0, 0.8 * w.u0[::-1]][:batch])
    plan = api.Plan.from_workload(w, precision=prec, batch=batch, col_kernel=col)
    assert plan.info()["col_kernel"] == col
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = _dev(u0 if batch > 1 else u0[0], dt)
    plan.advance(u, steps)
    got = u.double().cpu().numpy().reshape(batch, ny, nx)
    for i in range(batch):
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), np.ascontiguousarray(u0[i]), steps, threads=True)
        if prec == "fp64":
            assert rel_linf(got[i], ref) < 1e-11, i
        else:
            assert rel_l2(got[i], ref) < 1e-5, i


def test_kernel_choices_that_do_not_fit_are_refused():
    from paper_2103_06080_b300 import _lib as L
    api = _api()
    w = inputs.config(2, nx=64, ny=4096, n_steps=4)
    for prec, opt in (("fp32", dict(col_kernel="tma")), ("fp64", dict(col_kernel="pair")),
                      ("fp64", dict(row_kernel="pair")), ("fp32", dict(col_kernel="pair", fp32_state="plain"))):
        with pytest.raises(L.KzkError) as e:
            api.Plan.from_workload(w, precision=prec, **opt)
        assert e.value.status == L.KZK_ERR_SIZE, (prec, opt)
    with pytest.raises(ValueError):
        api.Plan.from_workload(w, precision="fp32", col_kernel="nope")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotuned_plan_matches_oracle(prec):
    """autotune=True times every fitting kernel combination at plan creation
    and keeps the fastest; whichever it keeps computes the same step."""
    api = _api()
    w = inputs.config(2, nx=512, ny=256, n_steps=20)
    plan = api.Plan.from_workload(w, precision=prec, autotune=True)
    info = plan.info()
    assert info["autotune"] and info["row_kernel"] in ("pair", "single") and info["col_kernel"] in ("pair", "tma", "tile")
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = _dev(w.u0, dt)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    got = u.double().cpu().numpy()
    if prec == "fp64":
        assert rel_linf(got, ref) < 1e-11, info
    else:
        assert rel_l2(got, ref) < 1e-5, info


# two relaxation processes (an extra diagonal term of the linear multiplier)
RELAX = dict(relax_C=(2e-4, 6e-4), relax_theta=(0.02, 0.1))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-7)])
def test_tables_with_relaxation_match_oracle(prec, tol):
    api = _api()
    w = inputs.config(1, nx=64, ny=32)
    plan = api.Plan.from_workload(w, precision=prec, **RELAX)
    E, P1, P2 = plan.tables()
    oE, oP1, oP2 = oracle.tables(oracle.Params(**inputs.oracle_params(w, **RELAX)))
    nl, nm = w.ny // 2 + 1, w.nx // 2 + 1
    for got, ref in ((E, oE), (P1, oP1), (P2, oP2)):
        ref = ref[:nl, :nm]
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        assert np.max(err[np.abs(ref) > 1e-280]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_relaxation_run_matches_oracle(prec):
    api = _api()
    w = inputs.config(2, nx=512, ny=64, n_steps=40)
    plan = api.Plan.from_workload(w, precision=prec, **RELAX)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = _dev(w.u0, dt)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w, **RELAX)), w.u0, w.n_steps, threads=True)
    plain = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_l2(plain, ref) > 1e-4          # the processes change the answer
    got = u.double().cpu().numpy()
    if prec == "fp64":
        assert rel_linf(got, ref) < 1e-11
    else:
        assert rel_l2(got, ref) < 1e-5


def test_relaxation_adjoint_matches_oracle():
    api = _api()
    w = inputs.config(2, nx=128, ny=32, n_steps=10)
    plan = api.Plan.from_workload(w, precision="fp64", **RELAX)
    p = oracle.Params(**inputs.oracle_params(w, **RELAX))
    g_end = 2 * w.dtau * oracle.run(p, w.u0, w.n_steps)
    ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    g0 = plan.adjoint(_dev(w.u0), _dev(g_end), w.n_steps, ckpt_every=3)
    assert rel_linf(g0.cpu().numpy(), ref) < 1e-10


def test_batch_instances_are_independent():
    api = _api()
    ws = [inputs.config(1, nx=128, ny=32) for _ in range(3)]
    u0 = np.stack([inputs.nwave(128, 32, a0=a, seed=s) for a, s in ((1.0, 1), (0.7, 2), (1.2, 3))])
    w = ws[0]
    plan = api.Plan.from_workload(w, precision="fp64", batch=3, lf_umax=1.5)
    u = _dev(u0)
    plan.advance(u, 7)
    for i in range(3):
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w, lf_umax=1.5)), u0[i], 7)
        assert rel_linf(u[i].cpu().numpy(), ref) < 1e-12


def test_extreme_sizes():
    api = _api()
    for nx, ny, steps in ((8, 2, 5), (8192, 2, 2), (16, 4096, 2)):
        w = inputs.config(1, nx=nx, ny=ny)
        plan = api.Plan.from_workload(w, precision="fp64")
        u = _dev(w.u0)
        plan.advance(u, steps)
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, steps, threads=True)
        assert rel_linf(u.cpu().numpy(), ref) < 1e-12, (nx, ny)


def test_runs_are_bitwise_deterministic():
    api = _api()
    w = inputs.config(1, nx=256, ny=128)
    plan = api.Plan.from_workload(w, precision="fp32")
    a = _dev(w.u0, torch.float32)
    b = a.clone()
    plan.advance(a, 10)
    plan.advance(b, 10)
    assert torch.equal(a, b)


def test_nonfinite_input_is_reported():
    api = _api()
    w = inputs.config(1, nx=64, ny=16)
    plan = api.Plan.from_workload(w, precision="fp64")
    u0 = w.u0.copy()
    u0[3, 5] = np.nan
    st, d = plan.advance(_dev(u0), 2, diag=True)
    assert st == 4 and d[0]["run_nonfinite"] > 0


def test_cfl_bound_violation_is_reported():
    api = _api()
    w = inputs.config(1, nx=64, ny=16)
    plan = api.Plan.from_workload(w, precision="fp64", lf_umax=0.5)
    st, d = plan.advance(_dev(w.u0), 1, diag=True)
    assert st == 3 and d[0]["run_max_abs"] > 0.5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-3)])
def test_adjoint_matches_oracle_adjoint(prec, tol):
    api = _api()
    w = inputs.config(2, nx=128, ny=32, n_steps=10)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = api.Plan.from_workload(w, precision=prec)
    p = oracle.Params(**inputs.oracle_params(w))
    u_end = oracle.run(p, w.u0, w.n_steps)
    g_end = 2 * w.dtau * u_end
    ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    g0 = plan.adjoint(_dev(w.u0, dt), _dev(g_end, dt), w.n_steps, ckpt_every=4)   # segments 4, 4, 2
    assert rel_linf(g0.double().cpu().numpy(), ref) < tol


@pytest.mark.parametrize("nx,ny,steps", [(4096, 8, 4), (8192, 4, 3)])
def test_adjoint_long_rows_match_oracle_adjoint(nx, ny, steps):
    # rows of 4096 and 8192 points: the FP64 adjoint row pass at 256 and 512
    # threads (the launch variant for longer rows than the 2048 of the
    # adjoint workload)
    api = _api()
    w = inputs.config(2, nx=nx, ny=ny, n_steps=steps)
    plan = api.Plan.from_workload(w, precision="fp64")
    p = oracle.Params(**inputs.oracle_params(w))
    u_end = oracle.run(p, w.u0, w.n_steps)
    g_end = 2 * w.dtau * u_end
    ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    g0 = plan.adjoint(_dev(w.u0), _dev(g_end), w.n_steps, ckpt_every=2)
    assert rel_linf(g0.double().cpu().numpy(), ref) < 1e-10


def test_adjoint_finite_differences_fp64():
    # central differences on seeded unit directions (FP64),
    # |ad - fd| <= 1e-6 max(|fd|, 0.1 |g0| / sqrt(N)) (fd_util.py: factorised
    # loss difference, adjoint projected on the perturbation actually applied).
    # h = 3e-4, where the difference is most accurate on this case (measured
    # sweep: ~1e-9 relative; with h = 1e-6 its own rounding is up to ~3e-6)
    from fd_util import central_fd_torch, fd_bound
    api = _api()
    w = inputs.config(4, nx=256, ny=64, n_steps=40)
    plan = api.Plan.from_workload(w, precision="fp64")
    u0 = _dev(w.u0)
    y = u0.clone()
    plan.advance(y, w.n_steps)
    g0 = plan.adjoint(u0, 2 * w.dtau * y, w.n_steps, ckpt_every=8)
    gen = torch.Generator(device="cpu").manual_seed(4)
    for _ in range(4):
        v = torch.randn(u0.shape, generator=gen, dtype=torch.float64).cuda()
        v /= v.norm()
        ad, fd = central_fd_torch(plan, u0, v, 3e-4, w.n_steps, w.dtau, g0)
        assert abs(ad - fd) <= fd_bound(1e-6, fd, float(g0.norm()), g0.numel()), (ad, fd)


# exponential Euler (Sec. 3.2): plan option method="expeuler"
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_expeuler_run_matches_oracle(prec):
    api = _api()
    w = inputs.config(2, nx=512, ny=128, n_steps=30)
    plan = api.Plan.from_workload(w, precision=prec, method="expeuler")
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = _dev(w.u0, dt)
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w, method=1)), w.u0, w.n_steps, threads=True)
    rk = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_l2(rk, ref) > 1e-4                 # a different scheme
    got = u.double().cpu().numpy()
    if prec == "fp64":
        assert rel_linf(got, ref) < 1e-11
    else:
        assert rel_l2(got, ref) < 1e-5


def test_expeuler_stages_and_adjoint():
    api = _api()
    w = inputs.config(2, nx=128, ny=32, n_steps=8)
    plan = api.Plan.from_workload(w, method="expeuler")
    p = oracle.Params(**inputs.oracle_params(w, method=1))
    us, un = plan.step_stages(_dev(w.u0))
    ref = oracle.run(p, w.u0, 1)
    assert rel_linf(un.cpu().numpy(), ref) < 1e-12 and torch.equal(us, un)
    g_end = 2 * w.dtau * oracle.run(p, w.u0, w.n_steps)
    g_ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    g0 = plan.adjoint(_dev(w.u0), _dev(g_end), w.n_steps, ckpt_every=3)
    assert rel_linf(g0.cpu().numpy(), g_ref) < 1e-10


# FP32 row passes: row pairs in packed FP32 (default) and single rows
# (row_kernel="single"); both against the oracle, and against each other.
@pytest.mark.parametrize("nx,ny,batch,medium", [(512, 256, 1, False), (64, 2, 3, False), (8192, 4, 1, False),
                                                (256, 64, 2, True)])
def test_fp32_row_pair_and_single_row(nx, ny, batch, medium):
    api = _api()
    if medium:
        w = inputs.medium_config(nx, ny, 20)
    else:
        w = inputs.config(3, nx=nx, ny=ny, n_steps=40)
    u0 = np.stack([w.u0 * (1.0 - 0.1 * i) for i in range(batch)])
    ref = np.stack([oracle.run(oracle.Params(**inputs.oracle_params(w)), np.ascontiguousarray(x), w.n_steps,
                               threads=True) for x in u0])
    got = {}
    for rk in ("pair", "single"):
        plan = api.Plan.from_workload(w, precision="fp32", batch=batch, row_kernel=rk)
        assert plan.info()["row_kernel"] == rk
        u = _dev(u0, torch.float32)
        st, d = plan.advance(u, w.n_steps, diag=True)
        assert st == 0
        got[rk] = (u.double().cpu().numpy(), plan.diag_history(w.n_steps))
        plan.close()
    for rk in ("pair", "single"):
        assert rel_l2(got[rk][0], ref) < 1e-5
    assert rel_l2(got["pair"][0], got["single"][0]) < 2e-6
    # per-step FP64 diagnostics of every row pair agree with the single rows
    assert np.allclose(got["pair"][1][:, :, 1], got["single"][1][:, :, 1], rtol=1e-5)


# FP32 state: compensated (default: the spectral state as hi + lo, the column
# passes transforming increments) and plain (fp32_state="plain").  Over the
# 2000 steps of the precision workload the compensated state keeps the FP32
# error within the 1e-5 goal, where the plain state accumulates the rounding
# of a full-state transform pair every step.
def test_fp32_compensated_state_2000_steps():
    # the precision workload as specified: 1024 x 512, 2000 steps, FP64 oracle
    api = _api()
    w = inputs.config(3, nx=1024, ny=512, n_steps=2000)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    err = {}
    for state in ("compensated", "plain"):
        plan = api.Plan.from_workload(w, precision="fp32", fp32_state=state)
        assert plan.info()["fp32_state"] == state
        u = _dev(w.u0, torch.float32)
        plan.advance(u, w.n_steps)
        err[state] = rel_l2(u.double().cpu().numpy(), ref)
        plan.close()
    assert err["compensated"] < 1e-5, err
    assert err["compensated"] < err["plain"], err


@pytest.mark.parametrize("method", ["exprk22", "expeuler"])
def test_fp32_compensated_state_short_runs(method):
    api = _api()
    w = inputs.config(2, nx=256, ny=64, n_steps=30)
    p = oracle.Params(**inputs.oracle_params(w, method=1 if method == "expeuler" else 0))
    ref = oracle.run(p, w.u0, w.n_steps)
    for state in ("compensated", "plain"):
        for col in ("auto", "tile"):
            plan = api.Plan.from_workload(w, precision="fp32", method=method, fp32_state=state, col_kernel=col)
            u = _dev(w.u0, torch.float32)
            plan.advance(u, w.n_steps)
            assert rel_l2(u.double().cpu().numpy(), ref) < 1e-5, (state, col)
            plan.close()


# kzk_advance from replayed step graphs (the default) against direct launches:
# the graphs' sigma-dependent values come from device memory, computed with
# the host's expressions, so the results and the diagnostics agree bit for bit
@pytest.mark.parametrize("prec,kind", [("fp64", "stratified"), ("fp32", "stratified"), ("fp64", "medium"),
                                       ("fp32", "medium"), ("fp64", "mixed"), ("fp32", "euler")])
def test_graph_replay_matches_direct_launches(prec, kind):
    api = _api()
    kw = {}
    if kind == "medium":
        w = inputs.medium_config(128, 64, 40)
    elif kind == "mixed":
        w = inputs.config(2, nx=56, ny=50, n_steps=40)
    else:
        w = inputs.config(2, nx=256, ny=256, n_steps=40)
        if kind == "euler":
            kw["method"] = "expeuler"
    dt = torch.float64 if prec == "fp64" else torch.float32
    plans = {g: api.Plan.from_workload(w, precision=prec, graph=g, **kw) for g in ("on", "off")}
    assert plans["on"].info()["graph"] == "on" and plans["off"].info()["graph"] == "off"
    for steps, sigma0 in ((37, 0.0), (5, 0.41 * w.n_steps * w.dt), (16, 0.8 * w.n_steps * w.dt)):
        res = {}
        for g, plan in plans.items():
            u = _dev(w.u0, dt)
            st, d = plan.advance(u, steps, sigma0=sigma0, diag=True)
            assert st == 0
            res[g] = (u, plan.diag_history(steps), d[0])
        assert torch.equal(res["on"][0], res["off"][0]), (steps, sigma0)
        assert np.array_equal(res["on"][1], res["off"][1])
        assert res["on"][2] == res["off"][2]
    for plan in plans.values():
        plan.close()


def test_graph_launches_are_counted():
    """kzk_launch_count counts every kernel a replayed graph runs: the same
    number as the direct launches of the same steps."""
    api = _api()
    w = inputs.config(2, nx=256, ny=128, n_steps=40)
    counts = {}
    for g in ("on", "off"):
        plan = api.Plan.from_workload(w, graph=g)
        u = _dev(w.u0)
        plan.advance(u, 2)                     # graphs captured on the first call
        torch.cuda.synchronize()
        n0 = api.launch_count()
        plan.advance(u, 21)
        counts[g] = api.launch_count() - n0
        plan.close()
    # per replay one kernel writes the chunk's sigma values (two replays: 16 + 5 x 1 = 6)
    assert counts["on"] == counts["off"] + 6, counts
