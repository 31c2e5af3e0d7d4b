"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds data generation only -- none of the method's arithmetic.
It produces the N-wave initial pressure profile of Sec. 4 (with the readings
used here: ``u0 = a0 * (-tau/L)`` on ``|tau| < L`` with tanh edges of width
``2 dtau``, modulated in y by ``exp(-y^2/16)``, plus seeded uniform noise of
relative amplitude 1e-2), the seeded cubic atmosphere profiles B(sigma),
A(sigma), the mode data of the random medium of Algorithm 1, and the
workload configurations (sizes, step counts, seeds).

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014):
output i of seed s is mix64(s + (i+1) * 0x9E3779B97F4A7C15), converted to
[0, 1) with the top 53 bits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` uint64 outputs of SplitMix64(seed), starting at output ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Workload:
    """One propagation: grid, coefficients, step size, step count and u0."""
    nx: int
    ny: int
    n_steps: int
    dt: float
    u0: np.ndarray
    tau_min: float = -4.0
    tau_max: float = 4.0
    y_min: float = -8.0
    y_max: float = 8.0
    B: float = 0.05
    A: float = 7e-6
    lf_umax: float = 1.0
    B_prof: tuple = (1.0, 0.0, 0.0, 0.0)
    A_prof: tuple = (1.0, 0.0, 0.0, 0.0)
    has_profile: bool = False
    precision: str = "fp64"
    L: float = 1.0
    a0: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)
    medium: "Medium | None" = None

    @property
    def dtau(self) -> float:
        return (self.tau_max - self.tau_min) / self.nx

    @property
    def dy(self) -> float:
        return (self.y_max - self.y_min) / self.ny


def nwave(nx: int, ny: int, L: float = 1.0, a0: float = 1.0, noise: float = 1e-2,
          seed: int = 1, y_gauss: bool = True, tau_min: float = -4.0, tau_max: float = 4.0,
          y_min: float = -8.0, y_max: float = 8.0, edge_cells: float = 2.0) -> np.ndarray:
    """N-wave u0[ny][nx]: a0 (-tau/L) on |tau| < L, tanh edges of width
    ``edge_cells * dtau``, times exp(-y^2/16), plus a0 * noise * U[-1, 1)
    drawn in row-major order."""
    dtau = (tau_max - tau_min) / nx
    dy = (y_max - y_min) / ny
    tau = tau_min + dtau * np.arange(nx)
    y = y_min + dy * np.arange(ny)
    w = edge_cells * dtau
    prof = a0 * (-tau / L) * 0.5 * (np.tanh((tau + L) / w) - np.tanh((tau - L) / w))
    ymod = np.exp(-y * y / 16.0) if y_gauss else np.ones(ny)
    u = ymod[:, None] * prof[None, :]
    if noise:
        xi = 2.0 * uniform01(seed, nx * ny).reshape(ny, nx) - 1.0
        u = u + a0 * noise * xi
    return np.ascontiguousarray(u)


def cubic_profile(seed: int, sigma_end: float, spread: float = 0.2):
    """Coefficients (c0..c3) of p(sigma) = c0 + c1 sigma + c2 sigma^2 + c3 sigma^3
    with p within [1 - spread, 1 + spread] on [0, sigma_end] (extremes reached
    exactly), drawn from the seed.  Returns (coeffs, max of p on the interval)."""
    r = 2.0 * uniform01(seed, 4) - 1.0            # q(s) = r0 + r1 s + r2 s^2 + r3 s^3
    q = np.polynomial.Polynomial(r)
    cand = [0.0, 1.0] + [float(x.real) for x in q.deriv().roots()
                         if abs(x.imag) < 1e-12 and 0.0 <= x.real <= 1.0]
    vals = np.array([q(s) for s in cand])
    qmax = float(np.max(np.abs(vals)))
    c_s = np.array([1.0, 0.0, 0.0, 0.0]) + spread * r / qmax   # p(s) in s = sigma / sigma_end
    pmax = float(np.max([np.polynomial.Polynomial(c_s)(s) for s in cand]))
    c_sigma = tuple(float(c_s[k] / sigma_end ** k) for k in range(4))
    return c_sigma, pmax


def cfl_dt(dtau: float, B_max: float, umax: float, cfl: float = 0.4) -> float:
    """Step size at WENO CFL number ``cfl``: B_max * umax * dt = cfl * dtau."""
    return cfl * dtau / (B_max * umax)


@dataclass
class Medium:
    """Modes of the random velocity field of Algorithm 1 (the field itself --
    the sums over modes at each (sigma, y) -- is evaluated by the solver and by
    the oracle).  Per mode: |K_n| lambda, theta_n (angle of K_n to the sigma
    axis), phi_n (phase), |U~(K_n)| / c0 (amplitude normalised by the sound
    speed)."""
    klam: np.ndarray
    theta: np.ndarray
    phase: np.ndarray
    amp: np.ndarray

    @property
    def n_modes(self) -> int:
        return len(self.klam)

    def bounds(self):
        """Upper bounds of |U_par| and |U_perp| (sums of the mode amplitudes)."""
        return (float(np.sum(np.abs(self.amp * np.sin(self.theta)))),
                float(np.sum(np.abs(self.amp * np.cos(self.theta)))))


def random_medium(seed: int, n_modes: int = 128, c0: float = 343.0, T0: float = 2e-2, sigma_u: float = 3.0,
                  kl_range=(0.1, 9.0)) -> Medium:
    """Mode data of Algorithm 1: phases phi_n and angles theta_n uniform in
    [0, 2 pi) (SplitMix64 draws: the n_modes phases, then the n_modes
    angles), wavenumbers equispaced in [K_min, K_max] = [0.1/L, 9/L] with
    L = 4 lambda and lambda = T0 c0, amplitudes sqrt(E(K_n) / N) from the
    Gaussian spectrum E(K) = sigma_u^2 K^3 L^4 exp(-(K L / 2)^2) / 8 (SI
    units as printed: K in 1/m, L in m), normalised by c0."""
    lam = T0 * c0
    L = 4.0 * lam
    r = uniform01(seed, 2 * n_modes)
    phase = 2.0 * np.pi * r[:n_modes]
    theta = 2.0 * np.pi * r[n_modes:]
    K = np.linspace(kl_range[0] / L, kl_range[1] / L, n_modes)
    E = 0.125 * sigma_u ** 2 * K ** 3 * L ** 4 * np.exp(-(K * L / 2.0) ** 2)
    amp = np.sqrt(E / n_modes) / c0
    return Medium(klam=K * lam, theta=theta, phase=phase, amp=amp)


def medium_config(nx: int = 4096, ny: int = 2048, n_steps: int = 500, seed: int = 6,
                  n_modes: int = 128) -> Workload:
    """N-wave through the random medium of Algorithm 1 (homogeneous B, A).
    The step follows the WENO CFL bound of both flux directions with the
    paper's estimate |U_par|, |U_perp| <= 0.05 (Sec. 2):
    dt (2 pi 0.05 + B max|u0|) <= 0.4 dtau and dt 0.05 <= 0.4 dy."""
    u0 = nwave(nx, ny, L=1.0, a0=1.0, seed=seed)
    umax = float(np.max(np.abs(u0)))
    med = random_medium(seed + 500, n_modes)
    dtau, dy = 8.0 / nx, 16.0 / ny
    dt = min(0.4 * dtau / (2.0 * np.pi * 0.05 + 0.05 * umax), 0.4 * dy / 0.05)
    return Workload(nx=nx, ny=ny, n_steps=n_steps, dt=dt, u0=u0, lf_umax=1.1 * umax, precision="fp64",
                    name="medium", medium=med)


def config(idx: int, nx: int | None = None, ny: int | None = None,
           n_steps: int | None = None) -> Workload:
    """The five synthetic workloads (1-based ``idx``); sizes may be overridden
    for scaled-down parity cases."""
    if idx in (1, 4):
        nx = nx or (512 if idx == 1 else 2048)
        ny = ny or (256 if idx == 1 else 1024)
        n = n_steps if n_steps is not None else (200 if idx == 1 else 1000)
        seed = 1 if idx == 1 else 4
        u0 = nwave(nx, ny, L=1.0, a0=1.0, seed=seed)
        umax = float(np.max(np.abs(u0)))
        dt = cfl_dt(8.0 / nx, 0.05, umax)
        return Workload(nx=nx, ny=ny, n_steps=n, dt=dt, u0=u0, lf_umax=1.1 * umax,
                        precision="fp64", name=f"config{idx}")
    if idx in (2, 3):
        nx = nx or 4096
        ny = ny or 2048
        n = n_steps if n_steps is not None else 2000
        seed = 2
        a0 = 0.5 + float(uniform01(seed + 1000, 1)[0])
        u0 = nwave(nx, ny, L=1.0, a0=a0, seed=seed)
        umax = float(np.max(np.abs(u0)))
        # profiles live on [0, sigma_end]; sigma_end follows from dt, which
        # uses the profile's bound 1 + spread, so there is no circularity
        dt = cfl_dt(8.0 / nx, 0.05 * 1.2, umax)
        sigma_end = n * dt if n > 0 else 1.0
        Bp, _ = cubic_profile(seed + 2000, sigma_end)
        Ap, _ = cubic_profile(seed + 3000, sigma_end)
        return Workload(nx=nx, ny=ny, n_steps=n, dt=dt, u0=u0, lf_umax=1.1 * umax,
                        B_prof=Bp, A_prof=Ap, has_profile=True, a0=a0,
                        precision="fp64" if idx == 2 else "fp32", name=f"config{idx}")
    raise ValueError(f"no single-instance workload {idx}")


def batched_config(seed: int = 5, count: int = 64, n_steps: int = 500,
                   nx_choices=(1024, 2048, 4096, 8192), ny_choices=(256, 512, 1024, 2048),
                   scale: int = 1) -> list:
    """Heterogeneous batch: per instance Nx, Ny, N-wave L in [0.5, 2], amplitude
    in [0.5, 1.5] and B/A profiles drawn from the seed (FP32 bulk).  ``scale``
    divides both sizes, for scaled-down parity runs."""
    out = []
    r = uniform01(seed, 8 * count).reshape(count, 8)
    for i in range(count):
        nx = nx_choices[min(int(r[i, 0] * len(nx_choices)), len(nx_choices) - 1)] // scale
        ny = ny_choices[min(int(r[i, 1] * len(ny_choices)), len(ny_choices) - 1)] // scale
        L = 0.5 + 1.5 * float(r[i, 2])
        a0 = 0.5 + float(r[i, 3])
        iseed = seed * 1000 + i
        u0 = nwave(nx, ny, L=L, a0=a0, seed=iseed)
        umax = float(np.max(np.abs(u0)))
        dt = cfl_dt(8.0 / nx, 0.05 * 1.2, umax)
        sigma_end = n_steps * dt if n_steps > 0 else 1.0
        Bp, _ = cubic_profile(iseed + 2000, sigma_end)
        Ap, _ = cubic_profile(iseed + 3000, sigma_end)
        out.append(Workload(nx=nx, ny=ny, n_steps=n_steps, dt=dt, u0=u0, lf_umax=1.1 * umax,
                            B_prof=Bp, A_prof=Ap, has_profile=True, precision="fp32",
                            L=L, a0=a0, name=f"batch{i}"))
    return out


def oracle_params(w: Workload, **over):
    """Keyword arguments describing ``w`` for the oracle's Params."""
    d = dict(nx=w.nx, ny=w.ny, dt=w.dt, tau_min=w.tau_min, tau_max=w.tau_max, y_min=w.y_min,
             y_max=w.y_max, B=w.B, A=w.A, lf_umax=w.lf_umax, B_prof=tuple(w.B_prof),
             A_prof=tuple(w.A_prof), has_profile=w.has_profile)
    if w.medium is not None:
        d.update(mode_klam=w.medium.klam, mode_theta=w.medium.theta, mode_phase=w.medium.phase,
                 mode_amp=w.medium.amp)
    d.update(over)
    return d


