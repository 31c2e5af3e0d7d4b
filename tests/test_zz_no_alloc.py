"""kzk_rhs_noalloc: the nonlinear term b(sigma, u) for callers that cannot let
the library allocate device memory (a process whose pool allocator owns all
device memory, or a latency-critical path that cannot take cudaMalloc's
implicit synchronisation).  Its scratch is a file-scope device array, so it
needs no plan.  The GPU test calls it through the C ABI twice in a row and
compares each result with kzk_rhs (the plan-based entry point) within the
tolerances the other parity tests use.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2103_06080_b300 import _lib as L
from paper_2103_06080_b300 import inputs


def _grid_coeffs(w, prec):
    g = L.KzkGrid(nx=w.nx, ny=w.ny, tau_min=w.tau_min, tau_max=w.tau_max, y_min=w.y_min, y_max=w.y_max,
                  prec=L.KZK_FP64 if prec == "fp64" else L.KZK_FP32)
    c = L.KzkCoeffs(B=w.B, A=w.A, lf_umax=w.lf_umax, B_prof=(ctypes.c_double * 4)(*w.B_prof),
                    A_prof=(ctypes.c_double * 4)(*w.A_prof), has_profile=int(w.has_profile))
    return g, c


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_cuda_available(), reason="host-only check (placeholder pointers)")
def test_noalloc_rejects_sizes_beyond_its_maximum():
    # checked on the host before any device work; the pointers are never used
    w = inputs.config(1, nx=1024, ny=512)           # 524288 points > 262144
    g, c = _grid_coeffs(w, "fp64")
    st = L.lib().kzk_rhs_noalloc(ctypes.byref(g), ctypes.byref(c), 1, ctypes.c_void_p(16), ctypes.c_void_p(32),
                                 0.0, None)
    assert st == L.KZK_ERR_SIZE
    assert b"KZK_NOALLOC_MAX_POINTS" in L.lib().kzk_last_error()
    w2 = inputs.config(1, nx=512, ny=256)
    g2, c2 = _grid_coeffs(w2, "fp64")
    st = L.lib().kzk_rhs_noalloc(ctypes.byref(g2), ctypes.byref(c2), 3, ctypes.c_void_p(16), ctypes.c_void_p(32),
                                 0.0, None)                  # batch 3: 393216 points
    assert st == L.KZK_ERR_SIZE


@pytest.mark.gpu
@pytest.mark.parametrize("prec,nx,ny,batch", [("fp64", 512, 256, 2), ("fp32", 256, 128, 1),
                                               # the limits of the fixed scratch layout: the longest row
                                               # (largest twiddle tables and shared-memory request) at
                                               # exactly KZK_NOALLOC_MAX_POINTS points, and FP32 batches
                                               ("fp64", 8192, 32, 1), ("fp32", 1024, 64, 4)])
def test_noalloc_rhs_matches_plan_rhs_on_two_calls(prec, nx, ny, batch):
    import torch

    from paper_2103_06080_b300 import api

    dt = torch.float64 if prec == "fp64" else torch.float32
    w = inputs.config(2, nx=nx, ny=ny, n_steps=100)
    plan = api.Plan.from_workload(w, precision=prec, batch=batch)
    g, c = _grid_coeffs(w, prec)
    stream = torch.cuda.current_stream()
    for call, sigma in enumerate((0.11 * w.n_steps * w.dt, 0.73 * w.n_steps * w.dt)):
        u0 = np.stack([inputs.nwave(nx, ny, a0=w.a0, seed=10 * call + i) for i in range(batch)])
        u = torch.tensor(u0, dtype=dt, device="cuda")
        b = torch.empty_like(u)
        st = L.lib().kzk_rhs_noalloc(ctypes.byref(g), ctypes.byref(c), batch, u.data_ptr(), b.data_ptr(),
                                     float(sigma), ctypes.c_void_p(stream.cuda_stream))
        assert st == L.KZK_OK, L.lib().kzk_last_error()
        ref = plan.rhs(u, sigma=sigma)
        torch.cuda.synchronize()
        got, want = b.double().cpu().numpy(), ref.double().cpu().numpy()
        if prec == "fp64":
            assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12
        else:
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5
    plan.close()


@pytest.mark.gpu
def test_noalloc_call_leaves_device_memory_untouched():
    """The property the entry point exists for: after a warm-up (the first call
    in the context looks up the array and loads the kernels), further calls
    change the device's free memory by nothing.  No tensor is created between
    the two readings."""
    import torch
    cases = []
    for prec, nx, ny in (("fp64", 512, 128), ("fp32", 2048, 64)):
        w = inputs.config(2, nx=nx, ny=ny, n_steps=50)
        g, c = _grid_coeffs(w, prec)
        dt = torch.float64 if prec == "fp64" else torch.float32
        u = torch.tensor(w.u0, dtype=dt, device="cuda")
        cases.append((g, c, u, torch.empty_like(u)))
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def call_all(sigma):
        for g, c, u, b in cases:
            st = L.lib().kzk_rhs_noalloc(ctypes.byref(g), ctypes.byref(c), 1, u.data_ptr(), b.data_ptr(), sigma, sp)
            assert st == L.KZK_OK, L.lib().kzk_last_error()

    call_all(0.1)                       # warm-up: set-up and kernel loading
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call_all(0.2)
    call_all(0.3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
