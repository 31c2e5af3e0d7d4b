"""Parity of the CUDA path with the FP64 oracle at the headline grid shape.

The FP64 stratified-atmosphere workload runs 4096 x 2048 (tau x y): its y
columns have 2048 points, which the FP64 column kernels take in tiles of two
columns with the radix schedule 8 * 8 * 8 * 4, and its rows 4096 points.
These tests run that exact shape (and a narrow grid with the same column
length and many column tiles) through kzk_advance, as the benchmark does,
and compare element by element with the oracle (Eq. 11 / Algorithm 2,
STEP 1-4): relative L-infinity within 1e-11 in FP64.
"""
import numpy as np
import pytest

import oracle
from paper_2103_06080_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("sigma_frac", [0.0, 0.61])
def test_headline_grid_fp64_matches_oracle(sigma_frac):
    """The full 4096 x 2048 stratified workload (B(sigma), A(sigma) cubic
    profiles over its 2000 steps), three steps from two points of the run:
    sigma0 = 0 and sigma0 = 0.61 sigma_end, where the profiles are away from
    their starting values."""
    from paper_2103_06080_b300 import api
    w = inputs.config(2)
    assert (w.nx, w.ny) == (4096, 2048)
    steps = 3
    sigma0 = sigma_frac * w.n_steps * w.dt
    plan = api.Plan.from_workload(w, precision="fp64")
    u = torch.tensor(w.u0, dtype=torch.float64, device="cuda")
    st, d = plan.advance(u, steps, sigma0=sigma0, diag=True)
    assert st == 0
    p = oracle.Params(**inputs.oracle_params(w))
    ref, hist = oracle.run(p, w.u0, steps, sigma0=sigma0, threads=True, want_hist=True)
    got = u.cpu().numpy()
    assert rel_linf(got, ref) < 1e-11
    # FP64 diagnostics of the final state against the oracle's
    od = oracle.diag(p, ref)
    assert abs(d[0]["energy"] - od[1]) < 1e-11 * od[1]
    assert abs(d[0]["max_abs"] - od[2]) < 1e-11 * od[2]
    plan.close()


def test_headline_grid_fp32_matches_oracle():
    """The FP32 precision form on the same grid (row pairs, column pairs,
    compensated state) for three steps: relative l2 within 1e-5."""
    from paper_2103_06080_b300 import api
    w = inputs.config(3)
    steps = 3
    plan = api.Plan.from_workload(w, precision="fp32")
    u = torch.tensor(w.u0, dtype=torch.float32, device="cuda")
    plan.advance(u, steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, steps, threads=True)
    assert rel_l2(u.double().cpu().numpy(), ref) < 1e-5
    plan.close()


def test_ny2048_many_column_tiles_fp64():
    """Column length 2048 in FP64 on 128 spectral columns (64 tiles of two),
    20 steps of the stratified recipe."""
    from paper_2103_06080_b300 import api
    w = inputs.config(2, nx=256, ny=2048, n_steps=20)
    plan = api.Plan.from_workload(w, precision="fp64")
    u = torch.tensor(w.u0, dtype=torch.float64, device="cuda")
    plan.advance(u, w.n_steps)
    ref = oracle.run(oracle.Params(**inputs.oracle_params(w)), w.u0, w.n_steps, threads=True)
    assert rel_linf(u.cpu().numpy(), ref) < 1e-11
    plan.close()
