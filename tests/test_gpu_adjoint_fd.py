"""The adjoint workload's finite-difference protocol (GPU).

Loss L(u0) = sum_y integral u(sigma_end, tau, y)^2 dtau = dtau sum u_end^2 on
the 2048 x 1024 grid, 1000 ExpRK22 steps (Eq. 5 / Eq. 11) from the seeded
N-wave, checkpoint every 32 steps.  The gradient g0 = dL/du0 from kzk_adjoint
(the hand-written transpose of the step) is checked along 16 seeded
directions v ~ N(0, I), |v| = 1, against central differences

    fd = (L(u0 + h v) - L(u0 - h v)) / (2 h)

evaluated in FP64 through the FP64 forward path (fd_util.py: the loss
difference summed in factorised form, the adjoint projected on the
perturbation actually applied).

The step h.  The difference carries a truncation error ~h^2 and the
rounding of the two forward runs divided by 2h.  Over 1000 steps with shocks
the rounding of the FP64 forward map is amplified strongly: with h = 1e-6 the
difference changes by ~1e-3 relative when h changes by 1 %, so at that step
it measures rounding, not the derivative.  A sweep h = 1e-2 ... 1e-7 on this
workload puts the accurate range at h = 3e-3 ... 1e-2 (difference to the
adjoint 4e-9 ... 2e-7 relative), and the check runs there, at h = 3e-3.

FP64: |ad - fd| <= 1e-6 max(|fd|, 0.1 |g0| / sqrt(N)) in every direction
(fd_util.fd_bound: relative to |fd| except in a direction nearly orthogonal to
g0).  FP32: the FP32 plan's adjoint (FP32 recompute of the forward states,
FP32 transposed step) against the same FP64 differences with the bound at
1e-3 (the FP32 state itself carries ~1e-5 relative error after these steps,
which moves the linearisation point), and the whole FP32 gradient within 1e-3
relative l2 of the FP64 one.
"""
import numpy as np
import pytest
from fd_util import central_fd_torch, fd_bound

from paper_2103_06080_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_DIR = 16
H = 3e-3
CKPT = 32


@pytest.fixture(scope="module")
def protocol():
    from paper_2103_06080_b300 import api
    w = inputs.config(4)
    assert (w.nx, w.ny, w.n_steps) == (2048, 1024, 1000)
    plan = api.Plan.from_workload(w, precision="fp64")
    u0 = torch.tensor(w.u0, dtype=torch.float64, device="cuda")
    y = u0.clone()
    plan.advance(y, w.n_steps)
    g0 = plan.adjoint(u0, 2 * w.dtau * y, w.n_steps, ckpt_every=CKPT)
    rng = np.random.default_rng(4)
    fd, ad, dirs = [], [], []
    for _ in range(N_DIR):
        v = torch.tensor(rng.standard_normal(w.u0.shape), dtype=torch.float64, device="cuda")
        v /= v.norm()
        a, f = central_fd_torch(plan, u0, v, H, w.n_steps, w.dtau, g0)
        ad.append(a)
        fd.append(f)
        dirs.append(((u0 + H * v) - (u0 - H * v)) / (2 * H))
    plan.close()
    return w, u0, g0, np.array(fd), np.array(ad), dirs


def test_adjoint_fd_protocol_fp64(protocol):
    w, u0, g0, fd, ad, _ = protocol
    rel = np.abs(ad - fd) / np.abs(fd)
    bound = np.array([fd_bound(1e-6, f, float(g0.norm()), g0.numel()) for f in fd])
    print(f"fp64 adjoint vs central FD (h = {H}), {N_DIR} directions: max rel {rel.max():.3e}, "
          f"median {np.median(rel):.3e}; |fd| in [{np.abs(fd).min():.3e}, {np.abs(fd).max():.3e}]")
    assert np.all(np.abs(ad - fd) <= bound), rel


def test_adjoint_fd_protocol_fp32(protocol):
    from paper_2103_06080_b300 import api
    w, u0, g0, fd, _, dirs = protocol
    plan = api.Plan.from_workload(w, precision="fp32")
    u32 = u0.float()
    y = u32.clone()
    plan.advance(y, w.n_steps)
    g32 = plan.adjoint(u32, 2 * w.dtau * y, w.n_steps, ckpt_every=CKPT).double()
    plan.close()
    ad32 = np.array([float((g32 * dx).sum()) for dx in dirs])
    rel = np.abs(ad32 - fd) / np.abs(fd)
    bound = np.array([fd_bound(1e-3, f, float(g0.norm()), g0.numel()) for f in fd])
    whole = float((g32 - g0).norm() / g0.norm())
    print(f"fp32 adjoint vs FP64 central FD: max rel {rel.max():.3e}, median {np.median(rel):.3e}; "
          f"whole gradient rel l2 vs fp64 {whole:.3e}")
    assert whole < 1e-3
    assert np.all(np.abs(ad32 - fd) <= bound), rel
