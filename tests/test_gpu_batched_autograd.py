"""Batched persistent launch and the autograd wrapper (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small_batch(precision):
    ws = inputs.batched_config(seed=5, count=4, n_steps=20, scale=8)   # Nx 128..1024, Ny 32..256
    for w in ws:
        w.precision = precision
    return ws


@pytest.mark.parametrize("prec,mode,state", [("fp64", "persistent", "auto"), ("fp32", "persistent", "compensated"),
                                              ("fp32", "persistent", "plain"), ("fp64", "streams", "auto"),
                                              ("fp32", "streams", "compensated"), ("fp32", "streams", "plain")])
def test_batched_matches_single_plans(prec, mode, state):
    from paper_2103_06080_b300 import api
    # the persistent kernel runs the per-tile column bodies and the
    # single-row bodies (FP32: with the compensated or the plain state):
    # compare with single plans on the same kernels, bit for bit; streams mode
    # runs the instances' own default kernels.  FP64 single plans on the
    # per-tile kernels carry the state's y-spectrum between steps (four
    # y-transforms per step, the persistent kernel five): the same step to
    # rounding, compared at 1e-13
    kw = dict(fp32_state=state) if prec == "fp32" else {}
    single = dict(row_kernel="single", col_kernel="tile") if mode == "persistent" else {}
    dt = torch.float64 if prec == "fp64" else torch.float32
    ws = _small_batch(prec)
    bp = api.BatchedPlan(ws, precision=prec, autotune=(mode == "persistent"), mode=mode, **kw)
    us = [torch.tensor(w.u0, dtype=dt, device="cuda") for w in ws]
    st, diags = bp.advance(us, 20, diag=True)
    assert st == 0
    for w, u, d in zip(ws, us, diags):
        p = api.Plan.from_workload(w, precision=prec, **kw, **single)
        v = torch.tensor(w.u0, dtype=dt, device="cuda")
        p.advance(v, 20)
        if prec == "fp64" and mode == "persistent":
            assert float((u - v).abs().max() / v.abs().max()) < 1e-13, (w.nx, w.ny)
        else:
            assert torch.equal(u, v), (w.nx, w.ny)
        assert np.isfinite(d["energy"]) and d["run_nonfinite"] == 0
        p.close()
    # a second call replays the captured graph
    bp.advance(us, 20, sigma0=20 * ws[0].dt)
    bp.close()


def test_batched_streams_autotuned_matches_oracle():
    """Streams mode with autotuned instances (each instance's kernel choice
    made by timing at creation) against the FP64 oracle."""
    from paper_2103_06080_b300 import api
    ws = _small_batch("fp32")[:3]
    bp = api.BatchedPlan(ws, precision="fp32", autotune=True, mode="streams")
    us = [torch.tensor(w.u0, dtype=torch.float32, device="cuda") for w in ws]
    bp.advance(us, 20)
    for w, u in zip(ws, us):
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 20, threads=True)
        got = u.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5, (w.nx, w.ny)
    bp.close()


def test_batched_fp32_persistent_accuracy():
    """The persistent launch carries the compensated FP32 state: against the
    FP64 oracle after 200 steps, relative l2 within 1e-5."""
    from paper_2103_06080_b300 import api
    # workloads whose atmosphere profiles span the 200 steps
    ws = inputs.batched_config(seed=5, count=4, n_steps=200, scale=8)[:2]
    bp = api.BatchedPlan(ws, precision="fp32", autotune=False, mode="persistent")
    us = [torch.tensor(w.u0, dtype=torch.float32, device="cuda") for w in ws]
    bp.advance(us, 200)
    for w, u in zip(ws, us):
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 200, threads=True)
        got = u.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5, (w.nx, w.ny)
    bp.close()


def test_batched_fp64_matches_oracle():
    from paper_2103_06080_b300 import api
    ws = _small_batch("fp64")[:2]
    bp = api.BatchedPlan(ws, precision="fp64", autotune=False, mode="persistent")
    us = [torch.tensor(w.u0, dtype=torch.float64, device="cuda") for w in ws]
    bp.advance(us, 10)
    for w, u in zip(ws, us):
        ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, 10, threads=True)
        got = u.cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-11


def test_batched_barrier_timeout_is_reported_and_recoverable():
    # every barrier waits for one CTA more than launched; the bounded wait runs
    # out (0.2 s), the kernel leaves and the call reports KZK_ERR_TIMEOUT
    from paper_2103_06080_b300 import _lib as L
    from paper_2103_06080_b300 import api
    ws = _small_batch("fp32")[:2]
    bp = api.BatchedPlan(ws, precision="fp32", autotune=False, mode="persistent")
    us = [torch.tensor(w.u0, dtype=torch.float32, device="cuda") for w in ws]
    bp.test_barrier(1, 200)
    with pytest.raises(L.KzkError) as e:
        bp.advance(us, 2)
    assert e.value.status == L.KZK_ERR_TIMEOUT
    bp.test_barrier(0, 2000)
    us = [torch.tensor(w.u0, dtype=torch.float32, device="cuda") for w in ws]
    bp.advance(us, 2)
    torch.cuda.synchronize()
    assert all(torch.isfinite(u).all() for u in us)


def test_autograd_gradient_matches_adjoint_and_oracle():
    from paper_2103_06080_b300 import api
    from paper_2103_06080_b300.autograd import advance
    w = inputs.config(2, nx=128, ny=32, n_steps=8)
    plan = api.Plan.from_workload(w, precision="fp64")
    u0 = torch.tensor(w.u0, dtype=torch.float64, device="cuda", requires_grad=True)
    u = advance(u0, plan, w.n_steps, 0.0, 3)
    loss = (u * u).sum() * w.dtau           # sum_y integral u^2 dtau
    loss.backward()
    p = oracle.Params(**inputs.oracle_params(w))
    u_end = oracle.run(p, w.u0, w.n_steps)
    ref = oracle.adjoint(p, w.u0, 2 * w.dtau * u_end, w.n_steps)
    g = u0.grad.cpu().numpy()
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-10
