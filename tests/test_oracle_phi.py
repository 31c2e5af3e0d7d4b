"""Pins of the oracle's phi-functions (Eq. 5 / Eq. 11) against high-precision
evaluation of their definitions, their limits at z = 0, and structural
properties of the tables (Hermitian symmetry, dissipativity)."""
import mpmath as mp
import numpy as np
import pytest

import oracle

mp.mp.dps = 50


def phi_mp(z):
    z = mp.mpc(z.real, z.imag)
    E = mp.exp(z)
    if z == 0:
        return complex(E), 1.0 + 0j, 0.5 + 0j
    P1 = (E - 1) / z
    P2 = (E - 1 - z) / z ** 2
    return complex(E), complex(P1), complex(P2)


SAMPLES = [1e-9 + 0j, 1e-4 - 2e-4j, 0.05 + 0.1j, -0.12 + 0.2j, 0.1 + 0j, -0.2499 + 0j, 0.2501j,
           0.3 - 0.3j, -0.45 + 0.1j, -1.0 + 0j, -3.0 + 7.0j, 0.5 + 0.5j, -40.0 + 200.0j,
           -1e6 + 0j, -1e15 + 0j, -2.0 - 150.0j, 1e-3j, -1e-12 + 1e-12j]


@pytest.mark.parametrize("z", SAMPLES)
def test_phi_matches_high_precision(z):
    E, P1, P2 = oracle.phi(z)
    rE, rP1, rP2 = phi_mp(z)
    for got, ref in ((E, rE), (P1, rP1), (P2, rP2)):
        scale = max(abs(ref), 1e-300)
        assert abs(got - ref) <= 4e-15 * scale + 1e-300, (z, got, ref)


def test_phi_limits_at_zero():
    E, P1, P2 = oracle.phi(0j)
    assert E == 1.0 and P1 == 1.0 and P2 == 0.5


def test_phi_series_and_quotient_agree_across_switch():
    # the switch between series and quotient sits at |z| = 0.25: both sides
    # of it must agree with the definition to full precision
    for ang in np.linspace(0, 2 * np.pi, 13):
        for r in (0.2499999, 0.2500001):
            z = r * np.exp(1j * ang)
            _, P1, P2 = oracle.phi(z)
            _, rP1, rP2 = phi_mp(z)
            assert abs(P1 - rP1) < 4e-15 and abs(P2 - rP2) < 4e-15


def test_phi1_equals_one_plus_z_phi2():
    for z in SAMPLES:
        _, P1, P2 = oracle.phi(z)
        assert abs(P1 - (1 + z * P2)) <= 1e-14 * max(1.0, abs(P1), abs(z * P2))


def _params(nx=16, ny=8, A=7e-6, dt=0.1):
    return oracle.Params(nx=nx, ny=ny, dt=dt, A=A)


def test_tables_hermitian_symmetric():
    # z(-k_tau, -k_y) = conj z(k_tau, k_y): real fields stay real (Eq. 11)
    p = _params()
    E, P1, P2 = oracle.tables(p)
    for T in (E, P1, P2):
        flipped = np.roll(T[::-1, ::-1], (1, 1), axis=(0, 1))
        assert np.allclose(flipped, np.conj(T), rtol=1e-14, atol=1e-300)


def test_tables_dissipative_and_pure_diffraction_unitary():
    p = _params(A=7e-6)
    E, _, _ = oracle.tables(p)
    assert np.all(np.abs(E) <= 1.0 + 1e-15)
    q = _params(A=0.0)
    E0, _, _ = oracle.tables(q)
    # with A = 0, every mode with k_tau != 0 (and not the tau-Nyquist, which
    # carries no diffraction) is advanced by a pure phase up to O(eps)
    mags = np.abs(E0[:, 1:q.nx // 2])
    assert np.allclose(mags, 1.0, atol=1e-14)
    # k_tau = 0 with k_y != 0 is annihilated by the regularised multiplier
    assert np.all(np.abs(E0[1:, 0]) == 0.0)
    assert E0[0, 0] == 1.0
