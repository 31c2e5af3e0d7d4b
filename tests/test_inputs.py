"""Pins of the seeded input generator where it evaluates a formula of the paper.

Both the oracle and the CUDA path consume the random medium's mode data, so a
mistake in the generator would pass every parity test.  The amplitudes of
Algorithm 1 (|U~(K_n)| = sqrt(E(|K_n|)/N) with the Gaussian energy spectrum of
Sec. 2, normalised by c0) and the equispaced wavenumbers are checked against
values worked by hand from those formulas (tests/golden/medium_spectrum.txt).
"""
import os

import numpy as np

from paper_2103_06080_b300 import inputs


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "medium_spectrum.txt")
    return np.loadtxt(path, ndmin=2)


def test_mode_amplitudes_match_hand_worked_spectrum():
    m = inputs.random_medium(506, n_modes=128)
    for n, klam, amp in _golden():
        n = int(n)
        assert abs(m.klam[n] - klam) <= 1e-15 * klam
        assert abs(m.amp[n] - amp) <= 1e-14 * amp, (n, m.amp[n], amp)


def test_wavenumbers_span_the_papers_interval():
    # |K_n| lambda from 0.1/4 to 9/4 (K in [0.1/L, 9/L], L = 4 lambda), equispaced
    m = inputs.random_medium(506, n_modes=128)
    assert abs(m.klam[0] - 0.025) < 1e-15 and abs(m.klam[-1] - 2.25) < 1e-15
    d = np.diff(m.klam)
    assert np.max(np.abs(d - d[0])) < 1e-15
    # angles and phases uniform in [0, 2 pi)
    assert np.all((m.theta >= 0) & (m.theta < 2 * np.pi))
    assert np.all((m.phase >= 0) & (m.phase < 2 * np.pi))
