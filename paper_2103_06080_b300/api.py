"""Python face of the CUDA propagator: a Plan wrapping the C ABI.

PyTorch supplies device memory and streams; all computation happens in
libkzk.so.  State tensors are CUDA tensors of shape [batch, ny, nx] (or
[ny, nx] for batch 1), contiguous, float64 for FP64 plans and float32 for
FP32 plans.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def make_options(row_kernel: str = "auto", col_kernel: str = "auto", fp32_state: str = "auto",
                 transforms: str = "auto", autotune: bool = False, graph: str = "auto") -> "L.KzkOptions":
    """kzk_options from names: row_kernel auto|pair|single, col_kernel
    auto|pair|tma|tile, fp32_state auto|compensated|plain, transforms
    auto|mixed, graph auto|on|off (advance from replayed step graphs);
    autotune times the open kernel choices at plan creation."""
    vals = {}
    for key, name in (("row_kernel", row_kernel), ("col_kernel", col_kernel), ("fp32_state", fp32_state),
                      ("transforms", transforms), ("graph", graph)):
        table = L.OPTION_VALUES[key]
        if name not in table:
            raise ValueError(f"{key} must be one of {sorted(table)}, got {name!r}")
        vals[key] = table[name]
    return L.KzkOptions(autotune=int(bool(autotune)), **vals)


def _option_names(o: "L.KzkOptions") -> dict:
    out = {}
    for key, table in L.OPTION_VALUES.items():
        inv = {v: k for k, v in table.items()}
        out[key] = inv.get(getattr(o, key), getattr(o, key))
    out["autotune"] = bool(o.autotune)
    return out


class Plan:
    """One plan: grid, coefficients and step dsigma shared by `batch` propagations."""

    def __init__(self, nx: int, ny: int, dt: float, precision: str = "fp64", batch: int = 1,
                 B: float = 0.05, A: float = 7e-6, lf_umax: float = 1.0,
                 tau_min: float = -4.0, tau_max: float = 4.0, y_min: float = -8.0, y_max: float = 8.0,
                 B_prof: Sequence[float] = (1.0, 0.0, 0.0, 0.0), A_prof: Sequence[float] = (1.0, 0.0, 0.0, 0.0),
                 has_profile: bool = False, diffraction: float = 0.0, reg_eps: float = 0.0,
                 weno_eps: float = 0.0, relax_C: Sequence[float] = (), relax_theta: Sequence[float] = (),
                 method: str = "exprk22", row_kernel: str = "auto", col_kernel: str = "auto",
                 fp32_state: str = "auto", transforms: str = "auto", autotune: bool = False,
                 graph: str = "auto"):
        if method not in ("exprk22", "expeuler"):
            raise ValueError("method must be 'exprk22' or 'expeuler'")
        if precision not in ("fp64", "fp32"):
            raise ValueError("precision must be 'fp64' or 'fp32'")
        self.nx, self.ny, self.dt, self.batch = int(nx), int(ny), float(dt), int(batch)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        g = L.KzkGrid(nx=self.nx, ny=self.ny, tau_min=tau_min, tau_max=tau_max, y_min=y_min, y_max=y_max,
                      prec=L.KZK_FP64 if precision == "fp64" else L.KZK_FP32)
        if len(relax_C) != len(relax_theta) or len(relax_C) > 2:
            raise ValueError("relax_C and relax_theta: equal lengths, at most 2 processes")
        pad = lambda v: (ctypes.c_double * 2)(*([float(x) for x in v] + [0.0] * (2 - len(v))))
        c = L.KzkCoeffs(B=B, A=A, diffraction=diffraction, reg_eps=reg_eps, weno_eps=weno_eps, lf_umax=lf_umax,
                        B_prof=(ctypes.c_double * 4)(*B_prof), A_prof=(ctypes.c_double * 4)(*A_prof),
                        has_profile=int(bool(has_profile)), n_relax=len(relax_C), relax_C=pad(relax_C),
                        relax_theta=pad(relax_theta),
                        method=L.KZK_EXPEULER if method == "expeuler" else L.KZK_EXPRK22)
        o = make_options(row_kernel, col_kernel, fp32_state, transforms, autotune, graph)
        self._grid, self._coeffs, self._opts = g, c, o
        h = ctypes.c_void_p()
        L.check(L.lib().kzk_plan_create_ex(ctypes.byref(g), ctypes.byref(c), self.dt, self.batch, ctypes.byref(o),
                                           ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_workload(cls, w, precision: Optional[str] = None, batch: int = 1, **over) -> "Plan":
        kw = dict(nx=w.nx, ny=w.ny, dt=w.dt, precision=precision or w.precision, batch=batch, B=w.B, A=w.A,
                  lf_umax=w.lf_umax, tau_min=w.tau_min, tau_max=w.tau_max, y_min=w.y_min, y_max=w.y_max,
                  B_prof=w.B_prof, A_prof=w.A_prof, has_profile=w.has_profile)
        kw.update(over)
        plan = cls(**kw)
        if getattr(w, "medium", None) is not None:
            plan.set_medium(w.medium)
        return plan

    def set_medium(self, medium) -> None:
        """Attach the random medium of Algorithm 1 (an object with arrays klam,
        theta, phase, amp per mode; None or zero modes removes it)."""
        if medium is None:
            m = L.KzkMedium(n_modes=0)
            L.check(L.lib().kzk_plan_set_medium(self.handle, ctypes.byref(m)))
            return
        arrs = [np.ascontiguousarray(getattr(medium, k), dtype=np.float64) for k in ("klam", "theta", "phase", "amp")]
        n = len(arrs[0])
        if any(a.shape != (n,) for a in arrs):
            raise ValueError("medium arrays must have one value per mode")
        P = ctypes.POINTER(ctypes.c_double)
        m = L.KzkMedium(n_modes=n, klam=arrs[0].ctypes.data_as(P), theta=arrs[1].ctypes.data_as(P),
                        phase=arrs[2].ctypes.data_as(P), amp=arrs[3].ctypes.data_as(P))
        L.check(L.lib().kzk_plan_set_medium(self.handle, ctypes.byref(m)))

    def medium_eval(self, sigma: float, stream=None):
        """(U_par, U_perp, dU_perp/dy) per row at sigma and max |U_perp|, as the kernels use them."""
        out = np.zeros((self.ny, 3))
        mx = ctypes.c_double()
        L.check(L.lib().kzk_medium_eval(self.handle, float(sigma), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(mx), _stream_ptr(stream)))
        return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy(), float(mx.value)

    def info(self) -> dict:
        """The kernel and state choices in effect (names as in make_options)."""
        o = L.KzkOptions()
        L.check(L.lib().kzk_plan_info(self.handle, ctypes.byref(o)))
        return _option_names(o)

    # -- helpers -------------------------------------------------------------
    def _check_state(self, t: torch.Tensor, name: str) -> None:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        want = self.batch * self.ny * self.nx
        if t.numel() != want or t.shape[-1] != self.nx or t.shape[-2] != self.ny:
            raise ValueError(f"{name} must have shape [{self.batch}, {self.ny}, {self.nx}], got {tuple(t.shape)}")

    @property
    def handle(self) -> int:
        if self._h is None or not self._h.value:
            raise RuntimeError("plan has been destroyed")
        return self._h.value

    # -- operations ----------------------------------------------------------
    def advance(self, u: torch.Tensor, n_steps: int, sigma0: float = 0.0, diag: bool = False,
                stream: Optional[torch.cuda.Stream] = None, raise_on_error: bool = True):
        """Advance u in place by n_steps ExpRK22 steps; with diag=True returns
        (status, [per-instance diagnostics dict])."""
        self._check_state(u, "u")
        d = (L.KzkDiag * self.batch)() if diag else None
        st = L.lib().kzk_advance(self.handle, u.data_ptr(), int(n_steps), float(sigma0), _stream_ptr(stream),
                                 d if diag else None)
        if diag:
            if raise_on_error and st not in (L.KZK_OK, L.KZK_ERR_CFL, L.KZK_ERR_NONFINITE):
                L.check(st)
            return st, [d[i].as_dict() for i in range(self.batch)]
        L.check(st)
        return None

    def diag_history(self, n: int, stream: Optional[torch.cuda.Stream] = None) -> np.ndarray:
        out = np.zeros((max(int(n), 1), self.batch, 4))
        L.check(L.lib().kzk_diag_history(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(n), _stream_ptr(stream)))
        return out[:n]

    def rhs(self, u: torch.Tensor, sigma: float = 0.0, stream=None) -> torch.Tensor:
        self._check_state(u, "u")
        b = torch.empty_like(u)
        L.check(L.lib().kzk_rhs(self.handle, u.data_ptr(), b.data_ptr(), float(sigma), _stream_ptr(stream)))
        return b

    def step_stages(self, u: torch.Tensor, sigma0: float = 0.0, stream=None):
        self._check_state(u, "u")
        us, un = torch.empty_like(u), torch.empty_like(u)
        L.check(L.lib().kzk_step_stages(self.handle, u.data_ptr(), us.data_ptr(), un.data_ptr(), float(sigma0),
                                        _stream_ptr(stream)))
        return us, un

    def tau_fft(self, x: torch.Tensor, direction: int, stream=None) -> torch.Tensor:
        """direction -1: physical [.., ny, nx] -> packed complex [.., ny, nx/2, 2];
        +1: the inverse."""
        if direction == -1:
            self._check_state(x, "x")
            out = torch.empty(x.shape[:-1] + (self.nx // 2, 2), dtype=self.dtype, device=x.device)
        else:
            if x.shape[-2:] != (self.nx // 2, 2) or not x.is_contiguous() or x.dtype != self.dtype:
                raise ValueError("packed spectrum must be contiguous [.., ny, nx/2, 2] of the plan dtype")
            out = torch.empty(x.shape[:-2] + (self.nx,), dtype=self.dtype, device=x.device)
        L.check(L.lib().kzk_tau_fft(self.handle, x.data_ptr(), out.data_ptr(), int(direction), _stream_ptr(stream)))
        return out

    def tables(self):
        """(E, Phi1, Phi2) as complex128 arrays [(ny/2+1), (nx/2+1)], unscaled."""
        shape = (self.ny // 2 + 1, self.nx // 2 + 1, 2)
        arrs = [np.zeros(shape) for _ in range(3)]
        P = ctypes.POINTER(ctypes.c_double)
        L.check(L.lib().kzk_get_tables(self.handle, *[a.ctypes.data_as(P) for a in arrs]))
        return tuple(a[..., 0] + 1j * a[..., 1] for a in arrs)

    def adjoint(self, u0: torch.Tensor, g_end: torch.Tensor, n_steps: int, sigma0: float = 0.0,
                ckpt_every: int = 32, stream=None) -> torch.Tensor:
        self._check_state(u0, "u0")
        self._check_state(g_end, "g_end")
        g0 = torch.empty_like(u0)
        L.check(L.lib().kzk_adjoint(self.handle, u0.data_ptr(), g_end.data_ptr(), g0.data_ptr(), int(n_steps),
                                    float(sigma0), int(ckpt_every), _stream_ptr(stream)))
        return g0

    def advance_checkpointed(self, u: torch.Tensor, n_steps: int, sigma0: float = 0.0, ckpt_every: int = 32,
                             stream=None) -> None:
        """advance() that keeps the adjoint's checkpoints in the plan."""
        self._check_state(u, "u")
        L.check(L.lib().kzk_advance_checkpointed(self.handle, u.data_ptr(), int(n_steps), float(sigma0),
                                                 int(ckpt_every), _stream_ptr(stream)))

    def adjoint_checkpointed(self, g_end: torch.Tensor, stream=None) -> torch.Tensor:
        """Adjoint of the last advance_checkpointed run of this plan."""
        self._check_state(g_end, "g_end")
        g0 = torch.empty_like(g_end)
        L.check(L.lib().kzk_adjoint_checkpointed(self.handle, g_end.data_ptr(), g0.data_ptr(), _stream_ptr(stream)))
        return g0

    def kernel_times(self, u: torch.Tensor, n_steps: int, sigma0: float = 0.0, stream=None) -> list:
        """Mean device ms of one launch of [row stage 1, column stage 1, row
        stage 2, column stage 2] over n_steps steps (advances u)."""
        self._check_state(u, "u")
        ms = (ctypes.c_double * 4)()
        L.check(L.lib().kzk_kernel_times(self.handle, u.data_ptr(), int(n_steps), float(sigma0),
                                         _stream_ptr(stream), ms))
        return [float(x) for x in ms]

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().kzk_plan_destroy(self._h.value)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _grid_coeffs(w, precision):
    g = L.KzkGrid(nx=w.nx, ny=w.ny, tau_min=w.tau_min, tau_max=w.tau_max, y_min=w.y_min, y_max=w.y_max,
                  prec=L.KZK_FP64 if precision == "fp64" else L.KZK_FP32)
    c = L.KzkCoeffs(B=w.B, A=w.A, lf_umax=w.lf_umax, B_prof=(ctypes.c_double * 4)(*w.B_prof),
                    A_prof=(ctypes.c_double * 4)(*w.A_prof), has_profile=int(bool(w.has_profile)))
    return g, c


class BatchedPlan:
    """Many independent propagations (own grid, coefficients and dsigma each)
    advanced by one graph launch per call: mode "streams" (default) -- every
    instance's own kernels on its own captured stream, concurrently; mode
    "persistent" -- one persistent cooperative kernel for all instances.
    Keyword options (fp32_state, row_kernel, ...) apply to every instance."""

    def __init__(self, workloads: Sequence, precision: str = "fp32", autotune: bool = True,
                 mode: str = "streams", **options):
        if mode not in ("persistent", "streams"):
            raise ValueError("mode must be 'persistent' or 'streams'")
        if precision not in ("fp64", "fp32"):
            raise ValueError("precision must be 'fp64' or 'fp32'")
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.shapes = [(w.ny, w.nx) for w in workloads]
        n = len(workloads)
        gs = (L.KzkGrid * n)()
        cs = (L.KzkCoeffs * n)()
        dts = (ctypes.c_double * n)()
        for i, w in enumerate(workloads):
            gs[i], cs[i] = _grid_coeffs(w, precision)
            dts[i] = w.dt
        h = ctypes.c_void_p()
        flags = (L.KZK_BATCH_AUTOTUNE if autotune else 0) | (L.KZK_BATCH_STREAMS if mode == "streams"
                                                             else L.KZK_BATCH_PERSISTENT)
        o = make_options(**options)
        L.check(L.lib().kzk_plan_create_batched_ex(gs, cs, dts, n, flags, ctypes.byref(o), ctypes.byref(h)))
        self.mode = mode
        self._h = h
        self.n = n

    @property
    def handle(self) -> int:
        if self._h is None or not self._h.value:
            raise RuntimeError("plan has been destroyed")
        return self._h.value

    def advance(self, us: Sequence[torch.Tensor], n_steps: int, sigma0: float = 0.0, diag: bool = False,
                stream=None):
        if len(us) != self.n:
            raise ValueError(f"need {self.n} states")
        for t, (ny, nx) in zip(us, self.shapes):
            if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != nx * ny:
                raise ValueError(f"state must be a contiguous CUDA {self.dtype} tensor of {ny}x{nx}")
        ptrs = (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in us])
        d = (L.KzkDiag * self.n)() if diag else None
        st = L.lib().kzk_advance_batched(self.handle, ptrs, int(n_steps), float(sigma0), _stream_ptr(stream),
                                         d if diag else None)
        if diag:
            if st not in (L.KZK_OK, L.KZK_ERR_CFL, L.KZK_ERR_NONFINITE):
                L.check(st)
            return st, [d[i].as_dict() for i in range(self.n)]
        L.check(st)
        return None

    def info(self) -> dict:
        g, c, sm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        L.check(L.lib().kzk_batch_info(self.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(sm)))
        return {"grid_ctas": g.value, "tile_cap": c.value, "smem_bytes": sm.value}

    def test_barrier(self, extra_blocks: int, timeout_ms: int) -> None:
        L.check(L.lib().kzk_batch_test_barrier(self.handle, int(extra_blocks), int(timeout_ms)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().kzk_plan_destroy(self._h.value)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(L.lib().kzk_launch_count())


def tile_copy_rate(n: int, ny: int, pattern: str = "strip", stream=None) -> float:
    """Bytes per second the tensor memory accelerator copies the FP32
    column-pass tiles at (n complex columns, ny rows): pattern "strip" (the
    column pairs' 16-byte rows) or "contiguous" (the same bytes per CTA as one
    run); no arithmetic."""
    pat = {"strip": L.KZK_COPY_STRIP, "contiguous": L.KZK_COPY_CONTIGUOUS}[pattern]
    out = ctypes.c_double()
    L.check(L.lib().kzk_tile_copy_rate(int(n), int(ny), pat, _stream_ptr(stream), ctypes.byref(out)))
    return float(out.value)


def alu_peak(precision: str = "fp64", stream=None) -> float:
    """Measured FMA throughput (FLOP/s) of the current device."""
    out = ctypes.c_double()
    L.check(L.lib().kzk_alu_peak(L.KZK_FP64 if precision == "fp64" else L.KZK_FP32, _stream_ptr(stream),
                                 ctypes.byref(out)))
    return float(out.value)
