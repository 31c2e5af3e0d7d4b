"""FP64 CPU oracle of the ExpRK22 / WENO5 / FFT scheme -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it, and it imports nothing from the CUDA package.

The arithmetic lives in ``kzk_oracle.c`` (plain C, FP64, built with
``-fno-fast-math -ffp-contract=off``); this module only marshals numpy arrays.
Every function follows a passage of Einkemmer, Ostermann & Residori,
arXiv:2103.06080:

* ``fft1d`` / ``fft2d``      -- the discrete Fourier transforms of Sec. 3.3
  (textbook radix-2, forward sign -1, inverse scaled by 1/N).
* ``phi``, ``tables``         -- E, Phi1, Phi2 and z_jk of Eq. 11.
* ``weno_parts``, ``weno_rhs``-- WENO5 on the gradient form of Eq. 7.
* ``rhs``                     -- b(sigma, V) of Eq. 3 (homogeneous medium) plus
  the absorption-deviation term of a sigma-varying A.
* ``run``                     -- ExpRK22 in Fourier space, Eq. 11 / Algorithm 2.
* ``adjoint``                 -- the exact transpose of ``run``'s step.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, definitions or brute force (none is "parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBS: dict = {}


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
        ("y_min", ctypes.c_double), ("y_max", ctypes.c_double),
        ("B", ctypes.c_double), ("A", ctypes.c_double),
        ("diffraction", ctypes.c_double), ("reg_eps", ctypes.c_double),
        ("weno_eps", ctypes.c_double), ("lf_umax", ctypes.c_double),
        ("B_prof", ctypes.c_double * 4), ("A_prof", ctypes.c_double * 4),
        ("has_profile", ctypes.c_int32), ("dt", ctypes.c_double),
        ("n_relax", ctypes.c_int32), ("relax_C", ctypes.c_double * 2), ("relax_theta", ctypes.c_double * 2),
        ("n_modes", ctypes.c_int32), ("mode_klam", ctypes.c_void_p), ("mode_theta", ctypes.c_void_p),
        ("mode_phase", ctypes.c_void_p), ("mode_amp", ctypes.c_void_p),
        ("method", ctypes.c_int32),
    ]

_MODE_FIELDS = ("mode_klam", "mode_theta", "mode_phase", "mode_amp")


@dataclass
class Params:
    """Grid, coefficients and step size of one propagation (FP64 oracle)."""
    nx: int
    ny: int
    dt: float
    tau_min: float = -4.0
    tau_max: float = 4.0
    y_min: float = -8.0
    y_max: float = 8.0
    B: float = 0.05
    A: float = 7e-6
    diffraction: float = 1.0 / (4.0 * np.pi)
    reg_eps: float = 2.0 ** -53
    weno_eps: float = 1e-6
    lf_umax: float = 1.0
    B_prof: tuple = (1.0, 0.0, 0.0, 0.0)
    A_prof: tuple = (1.0, 0.0, 0.0, 0.0)
    has_profile: bool = False
    relax_C: tuple = ()          # relaxation strengths C_r (at most two processes)
    relax_theta: tuple = ()      # relaxation times theta_r (tau units), same length
    # random medium (Algorithm 1): per mode |K_n| lambda, theta_n, phi_n, |U~_n| / c0
    mode_klam: object = None
    mode_theta: object = None
    mode_phase: object = None
    mode_amp: object = None
    method: int = 0              # 0: ExpRK22 (Eq. 5); 1: exponential Euler (Sec. 3.2)

    def c(self) -> _Params:
        p = _Params()
        self._mode_arrays = []
        n_modes = 0 if self.mode_klam is None else len(self.mode_klam)
        for name, _ in _Params._fields_:
            if name == "n_relax":
                p.n_relax = len(self.relax_C)
                continue
            if name == "n_modes":
                p.n_modes = n_modes
                continue
            if name in _MODE_FIELDS:
                if n_modes:
                    a = np.ascontiguousarray(getattr(self, name), dtype=np.float64)
                    if a.shape != (n_modes,):
                        raise ValueError(f"{name}: expected {n_modes} values")
                    self._mode_arrays.append(a)          # kept alive with the Params
                    setattr(p, name, a.ctypes.data)
                continue
            v = getattr(self, name)
            if name in ("B_prof", "A_prof"):
                arr = (ctypes.c_double * 4)(*[float(x) for x in v])
                setattr(p, name, arr)
            elif name in ("relax_C", "relax_theta"):
                if len(v) > 2 or len(self.relax_C) != len(self.relax_theta):
                    raise ValueError("relax_C and relax_theta: equal lengths, at most 2")
                setattr(p, name, (ctypes.c_double * 2)(*([float(x) for x in v] + [0.0] * (2 - len(v)))))
            elif name in ("nx", "ny", "has_profile", "method"):
                setattr(p, name, int(v))
            else:
                setattr(p, name, float(v))
        return p


def _lib(threads: bool = False):
    key = "omp" if threads else "seq"
    if key not in _LIBS:
        name = "liboracle_omp.so" if threads else "liboracle.so"
        path = os.path.join(_HERE, name)
        if not os.path.exists(path):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_Params)
        lib.orc_fft1d.argtypes = [D, D, ctypes.c_int, ctypes.c_int]
        lib.orc_fft2d.argtypes = [D, D, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_phi.argtypes = [ctypes.c_double, ctypes.c_double, D]
        lib.orc_tables.argtypes = [P, D, D, D, D, D, D]
        lib.orc_weno_parts.argtypes = [D, ctypes.c_double, D, D, D]
        lib.orc_weno_grad.argtypes = [D, ctypes.c_double, D]
        lib.orc_weno_rhs.argtypes = [P, D, ctypes.c_double, D]
        lib.orc_weno_rhs_T.argtypes = [P, D, ctypes.c_double, D, D]
        lib.orc_rhs.argtypes = [P, D, ctypes.c_double, D]
        lib.orc_diag.argtypes = [P, D, D]
        lib.orc_run.argtypes = [P, D, ctypes.c_int64, ctypes.c_double, D, D]
        lib.orc_run_timed.argtypes = [P, D, ctypes.c_int64, ctypes.c_double, D]
        lib.orc_adjoint.argtypes = [P, D, D, ctypes.c_int64, ctypes.c_double, D]
        lib.orc_medium.argtypes = [P, ctypes.c_double, D, D, D]
        lib.orc_B_of.argtypes = [P, ctypes.c_double]
        lib.orc_B_of.restype = ctypes.c_double
        lib.orc_A_of.argtypes = [P, ctypes.c_double]
        lib.orc_A_of.restype = ctypes.c_double
        lib.orc_num_threads.restype = ctypes.c_int
        _LIBS[key] = lib
    return _LIBS[key]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads(threads: bool = True) -> int:
    return int(_lib(threads).orc_num_threads())


def fft1d(x, inverse: bool = False) -> np.ndarray:
    """Radix-2 DFT of a complex vector (forward sign -1; inverse scaled 1/N)."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    _lib().orc_fft1d(_ptr(re), _ptr(im), re.size, int(inverse))
    return re + 1j * im


def fft2d(x, inverse: bool = False, threads: bool = False) -> np.ndarray:
    """2-D transform of a [ny][nx] complex array, along tau then y."""
    x = np.asarray(x, dtype=np.complex128)
    ny, nx = x.shape
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    _lib(threads).orc_fft2d(_ptr(re), _ptr(im), nx, ny, int(inverse))
    return re + 1j * im


def phi(z: complex):
    """(E, Phi1, Phi2) at one complex z (Eq. 11)."""
    out = np.zeros(6)
    _lib().orc_phi(float(np.real(z)), float(np.imag(z)), _ptr(out))
    return complex(out[0], out[1]), complex(out[2], out[3]), complex(out[4], out[5])


def tables(p: Params, threads: bool = False):
    """Full [ny][nx] complex tables E, Phi1, Phi2 of Eq. 11."""
    shape = (p.ny, p.nx)
    arrs = [np.zeros(shape) for _ in range(6)]
    cp = p.c()
    _lib(threads).orc_tables(ctypes.byref(cp), *[_ptr(a) for a in arrs])
    return (arrs[0] + 1j * arrs[1], arrs[2] + 1j * arrs[3], arrs[4] + 1j * arrs[5])


def weno_parts(v, eps: float = 1e-6):
    """(q[3], beta[3], F) of one WENO5 interface from v_{-2..2}."""
    v = _f64(v)
    q, b, f = np.zeros(3), np.zeros(3), np.zeros(1)
    _lib().orc_weno_parts(_ptr(v), eps, _ptr(q), _ptr(b), _ptr(f))
    return q, b, float(f[0])


def weno_grad(v, eps: float = 1e-6) -> np.ndarray:
    v = _f64(v)
    g = np.zeros(5)
    _lib().orc_weno_grad(_ptr(v), eps, _ptr(g))
    return g


def medium(p: Params, sigma: float):
    """U_par, U_perp and d U_perp / dy at (sigma, y_j) for every row (Algorithm 1)."""
    a, b, c = (np.zeros(p.ny) for _ in range(3))
    cp = p.c()
    _lib().orc_medium(ctypes.byref(cp), float(sigma), _ptr(a), _ptr(b), _ptr(c))
    return a, b, c


def weno_rhs(p: Params, u, sigma: float = 0.0, threads: bool = False) -> np.ndarray:
    u = _f64(u).reshape(p.ny, p.nx)
    b = np.zeros_like(u)
    cp = p.c()
    _lib(threads).orc_weno_rhs(ctypes.byref(cp), _ptr(u), sigma, _ptr(b))
    return b


def weno_rhs_T(p: Params, u, mu, sigma: float = 0.0, threads: bool = False) -> np.ndarray:
    u = _f64(u).reshape(p.ny, p.nx)
    mu = _f64(mu).reshape(p.ny, p.nx)
    out = np.zeros_like(u)
    cp = p.c()
    _lib(threads).orc_weno_rhs_T(ctypes.byref(cp), _ptr(u), sigma, _ptr(mu), _ptr(out))
    return out


def rhs(p: Params, u, sigma: float = 0.0, threads: bool = False) -> np.ndarray:
    """b(sigma, u) in physical space (WENO part + absorption deviation)."""
    u = _f64(u).reshape(p.ny, p.nx)
    b = np.zeros_like(u)
    cp = p.c()
    _lib(threads).orc_rhs(ctypes.byref(cp), _ptr(u), sigma, _ptr(b))
    return b


def diag(p: Params, u) -> np.ndarray:
    """[mean, energy, max|u|, non-finite count]."""
    u = _f64(u).reshape(p.ny, p.nx)
    out = np.zeros(4)
    cp = p.c()
    _lib().orc_diag(ctypes.byref(cp), _ptr(u), _ptr(out))
    return out


def run(p: Params, u0, n_steps: int, sigma0: float = 0.0, threads: bool = False,
        want_ustar: bool = False, want_hist: bool = False):
    """Advance u0 by n_steps steps of p.method (ExpRK22 or exponential Euler).
    Returns u (and V* of the last step,
    and the [n_steps][4] diagnostics history when asked)."""
    u = _f64(u0).reshape(p.ny, p.nx).copy()
    us = np.zeros_like(u) if want_ustar else None
    hist = np.zeros((max(n_steps, 1), 4)) if want_hist else None
    cp = p.c()
    _lib(threads).orc_run(ctypes.byref(cp), _ptr(u), int(n_steps), float(sigma0),
                          _ptr(us) if us is not None else None,
                          _ptr(hist) if hist is not None else None)
    out = [u]
    if want_ustar:
        out.append(us)
    if want_hist:
        out.append(hist[:n_steps])
    return out[0] if len(out) == 1 else tuple(out)


def run_timed(p: Params, u0, n_steps: int, sigma0: float = 0.0, threads: bool = True):
    """(u after n_steps, wall seconds of each step; table set-up excluded)."""
    u = _f64(u0).reshape(p.ny, p.nx).copy()
    sec = np.zeros(max(int(n_steps), 1))
    cp = p.c()
    _lib(threads).orc_run_timed(ctypes.byref(cp), _ptr(u), int(n_steps), float(sigma0), _ptr(sec))
    return u, sec[:n_steps]


def adjoint(p: Params, u0, g_end, n_steps: int, sigma0: float = 0.0, threads: bool = False):
    """Gradient w.r.t. u0 of a loss whose gradient w.r.t. u(sigma_end) is g_end."""
    u0 = _f64(u0).reshape(p.ny, p.nx)
    g_end = _f64(g_end).reshape(p.ny, p.nx)
    g0 = np.zeros_like(u0)
    cp = p.c()
    _lib(threads).orc_adjoint(ctypes.byref(cp), _ptr(u0), _ptr(g_end), int(n_steps), float(sigma0), _ptr(g0))
    return g0


def B_of(p: Params, sigma: float) -> float:
    cp = p.c()
    return float(_lib().orc_B_of(ctypes.byref(cp), sigma))


def A_of(p: Params, sigma: float) -> float:
    cp = p.c()
    return float(_lib().orc_A_of(ctypes.byref(cp), sigma))
