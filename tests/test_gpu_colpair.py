"""The FP32 column passes on column pairs (kzk_colpair.cuh): every
supported length ny = 256 .. 4096, batches, both stages of the step, the
packed column 0, the exponential Euler step (output over its input), the
random medium, and agreement with the Stockham tile kernels they replace
(col_kernel="tma").  FP32 against the FP64 oracle: relative l2 within 1e-5."""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _api():
    from paper_2103_06080_b300 import api
    return api


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run32(w, u0, steps, batch=1, **kw):
    api = _api()
    plan = api.Plan.from_workload(w, precision="fp32", batch=batch, **kw)
    u = torch.tensor(np.ascontiguousarray(u0), dtype=torch.float32, device="cuda")
    plan.advance(u, steps)
    out = u.double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("nx,ny,steps", [(64, 256, 20), (32, 512, 20), (64, 1024, 16), (16, 2048, 12),
                                         (8, 4096, 8), (256, 256, 30)])
def test_colpair_runs_match_oracle(nx, ny, steps):
    w = inputs.config(2, nx=nx, ny=ny, n_steps=steps)
    got = _run32(w, w.u0, steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, steps, threads=True)
    assert rel_l2(got, ref) < 1e-5


def test_colpair_batch_of_two():
    w = inputs.config(2, nx=64, ny=512, n_steps=15)
    u0 = np.stack([w.u0, 0.7 * w.u0[::-1]])
    got = _run32(w, u0, 15, batch=2)
    p = oracle.Params(**inputs.oracle_params(w))
    for i in range(2):
        assert rel_l2(got[i], oracle.run(p, np.ascontiguousarray(u0[i]), 15, threads=True)) < 1e-5, i


@pytest.mark.parametrize("ny", [256, 2048])
def test_colpair_agrees_with_stockham_kernels(ny):
    w = inputs.config(2, nx=128, ny=ny, n_steps=20)
    a = _run32(w, w.u0, 20, col_kernel="pair")
    b = _run32(w, w.u0, 20, col_kernel="tma")
    assert rel_l2(a, b) < 1e-6
    assert np.max(np.abs(a - b)) > 0   # different kernels: the switch took effect


def test_colpair_one_step_stages():
    api = _api()
    w = inputs.config(2, nx=128, ny=512, n_steps=1)
    plan = api.Plan.from_workload(w, precision="fp32")
    s0 = 3 * w.dt
    us, un = plan.step_stages(torch.tensor(w.u0, dtype=torch.float32, device="cuda"), sigma0=s0)
    ref_un, ref_us = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 1, sigma0=s0, want_ustar=True)
    assert rel_l2(us.double().cpu().numpy(), ref_us) < 1e-6
    assert rel_l2(un.double().cpu().numpy(), ref_un) < 1e-6


def test_colpair_exponential_euler():
    w = inputs.config(2, nx=64, ny=256, n_steps=25)
    got = _run32(w, w.u0, 25, method="expeuler")
    p = oracle.Params(**inputs.oracle_params(w, method=1))
    assert rel_l2(got, oracle.run(p, w.u0, 25, threads=True)) < 1e-5


def test_colpair_random_medium():
    api = _api()
    w = inputs.medium_config(128, 256, 10)
    plan = api.Plan.from_workload(w, precision="fp32")
    u = torch.tensor(w.u0, dtype=torch.float32, device="cuda")
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_l2(u.double().cpu().numpy(), ref) < 1e-5


def test_colpair_diagnostics():
    """The per-step diagnostics reduced by the first column pair of each
    instance agree with the FP64 plan's."""
    api = _api()
    w = inputs.config(2, nx=64, ny=1024, n_steps=6)
    d = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        plan = api.Plan.from_workload(w, precision=prec)
        u = torch.tensor(w.u0, dtype=dt, device="cuda")
        plan.advance(u, w.n_steps, diag=True)
        d[prec] = plan.diag_history(w.n_steps)
        plan.close()
    assert np.all(np.isfinite(d["fp32"]))
    e32, e64 = d["fp32"][:, 0, 1], d["fp64"][:, 0, 1]
    assert np.max(np.abs(e32 - e64) / np.abs(e64)) < 1e-5


def test_colpair_with_relaxation():
    """Two relaxation processes change the tables only; the pair tables are
    built from them."""
    relax = dict(relax_C=(2e-4, 6e-4), relax_theta=(0.02, 0.1))
    w = inputs.config(2, nx=64, ny=512, n_steps=20)
    got = _run32(w, w.u0, 20, **relax)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w, **relax)), w.u0, 20, threads=True)
    plain = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 20, threads=True)
    assert rel_l2(plain, ref) > 1e-4
    assert rel_l2(got, ref) < 1e-5


def test_colpair_in_the_adjoint_recompute():
    """The FP32 adjoint recomputes each checkpoint segment with the forward
    step (column pairs at ny = 256); the gradient against the oracle's
    adjoint within the FP32 adjoint tolerance of the other grids (3e-3)."""
    api = _api()
    w = inputs.config(2, nx=64, ny=256, n_steps=8)
    plan = api.Plan.from_workload(w, precision="fp32")
    p = oracle.Params(**inputs.oracle_params(w))
    g_end = 2 * w.dtau * oracle.run(p, w.u0, w.n_steps)
    ref = oracle.adjoint(p, w.u0, g_end, w.n_steps)
    g0 = plan.adjoint(torch.tensor(w.u0, dtype=torch.float32, device="cuda"),
                      torch.tensor(g_end, dtype=torch.float32, device="cuda"), w.n_steps, ckpt_every=3)
    got = g0.double().cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 3e-3


def test_colpair_with_single_row_passes():
    """row_kernel="single": the single-row passes store b2 itself, and the
    column-pair stage 2 forms b2 - b1 from its two tiles."""
    w = inputs.config(2, nx=128, ny=512, n_steps=15)
    a = _run32(w, w.u0, 15, row_kernel="pair", col_kernel="pair")
    b = _run32(w, w.u0, 15, row_kernel="single", col_kernel="pair")
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 15, threads=True)
    assert rel_l2(b, ref) < 1e-5
    assert rel_l2(a, b) < 1e-6


@pytest.mark.parametrize("pattern", ["strip", "contiguous"])
def test_tile_copy_rate_is_a_plausible_bandwidth(pattern):
    # the ceiling the column passes' tile copies are compared with: a finite
    # rate between 0.1 and 20 TB/s for the 4096 x 2048 FP32 tiles
    from paper_2103_06080_b300 import api
    r = api.tile_copy_rate(2048, 2048, pattern)
    assert np.isfinite(r) and 1e11 < r < 2e13
