"""Pins of the oracle's WENO5 (Sec. 3.3, Eq. 7; Jiang-Shu weights, global
Lax-Friedrichs splitting) against the definitions the formulas come from:
polynomial reconstruction from cell averages, the Jiang-Shu smoothness
integral, the optimal linear weights, 5th-order convergence, conservation
and the analytic gradient."""
import numpy as np
import pytest
import sympy as sp

import oracle

x = sp.symbols("x")


def _reconstruction(cells):
    """Quadratic/quartic polynomial with the given cell averages over cells
    [i - 1/2, i + 1/2] (i in ``cells``, unit width), as sympy expression in x
    with symbolic averages v_i."""
    deg = len(cells) - 1
    cs = sp.symbols(f"c0:{deg + 1}")
    p = sum(c * x ** k for k, c in enumerate(cs))
    vs = {i: sp.Symbol(f"v{i}".replace("-", "m")) for i in range(-2, 3)}
    eqs = [sp.integrate(p, (x, i - sp.Rational(1, 2), i + sp.Rational(1, 2))) - vs[i] for i in cells]
    sol = sp.solve(eqs, cs)
    return p.subs(sol), vs


@pytest.fixture(scope="module")
def definitions():
    stencils = [[-2, -1, 0], [-1, 0, 1], [0, 1, 2]]
    q_exprs, b_exprs = [], []
    for st in stencils:
        p, vs = _reconstruction(st)
        q_exprs.append(sp.expand(p.subs(x, sp.Rational(1, 2))))
        # Jiang-Shu: beta = sum_l int_{cell 0} (d^l p / dx^l)^2 dx (unit width)
        beta = sum(sp.integrate(sp.diff(p, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
                   for l in (1, 2))
        b_exprs.append(sp.expand(beta))
    P5, vs = _reconstruction([-2, -1, 0, 1, 2])
    q5 = sp.expand(P5.subs(x, sp.Rational(1, 2)))
    d = sp.symbols("d0:3")
    eqs = sp.Poly(sum(di * qi for di, qi in zip(d, q_exprs)) - q5, *vs.values()).coeffs()
    dsol = sp.solve(eqs, d)
    syms = [vs[i] for i in range(-2, 3)]
    return ([sp.lambdify(syms, e) for e in q_exprs], [sp.lambdify(syms, e) for e in b_exprs],
            [float(dsol[di]) for di in d])


def test_candidates_and_indicators_match_definitions(definitions):
    qf, bf, _ = definitions
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.standard_normal(5)
        q, beta, _ = oracle.weno_parts(v)
        for r in range(3):
            assert abs(q[r] - qf[r](*v)) < 1e-13
            assert abs(beta[r] - bf[r](*v)) < 1e-12


def test_linear_weights_are_the_optimal_ones(definitions):
    qf, _, d = definitions
    assert np.allclose(d, [0.1, 0.6, 0.3], rtol=0, atol=1e-15)
    # with huge eps the weights collapse to d: the 5-point reconstruction
    rng = np.random.default_rng(1)
    v = rng.standard_normal(5)
    _, _, F = oracle.weno_parts(v, eps=1e30)
    assert abs(F - sum(di * qf[r](*v) for r, di in enumerate(d))) < 1e-13


def _params(nx, B=0.05, M=2.0, eps=1e-6, ny=1, L=2 * np.pi):
    return oracle.Params(nx=nx, ny=ny, dt=0.0, tau_min=0.0, tau_max=L, y_min=0.0, y_max=1.0,
                         B=B, lf_umax=M, weno_eps=eps)


def test_constant_state_gives_zero_rhs():
    p = _params(64, ny=4)
    b = oracle.weno_rhs(p, np.full((4, 64), 0.7312))
    assert np.all(b == 0.0)


def test_rhs_sums_to_zero_conservation():
    rng = np.random.default_rng(2)
    p = _params(128, ny=8)
    u = rng.standard_normal((8, 128))
    b = oracle.weno_rhs(p, u)
    assert np.max(np.abs(b.sum(axis=1))) < 1e-11 * np.max(np.abs(b))


def _order(eps, norm, ns=(32, 64, 128, 256)):
    errs = []
    for n in ns:
        p = _params(n, eps=eps)
        t = 2 * np.pi * np.arange(n) / n
        u = 0.5 + np.sin(t)
        exact = 0.5 * p.B * 2.0 * u * np.cos(t)          # (B/2) d_tau u^2
        e = oracle.weno_rhs(p, u[None, :])[0] - exact
        errs.append(np.max(np.abs(e)) if norm == "inf" else np.mean(np.abs(e)))
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_fifth_order_with_linear_weights():
    # l1 error against (B/2) d_tau u^2 on a smooth periodic profile; the
    # pre-asymptotic rates approach 5 from above, the last two are at 5
    rates = _order(1e30, "l1", ns=(64, 128, 256, 512))
    assert all(abs(r - 5.0) < 0.05 for r in rates[1:]), rates


def test_high_order_with_jiang_shu_weights():
    # JS weights lose order near critical points at moderate N; the mean rate
    # in l1 must still approach 5 (documented reading)
    rates = _order(1e-6, "l1")
    assert rates[-1] > 4.5, rates


def test_upwinding_of_split_fluxes_is_monotone_at_a_jump():
    # a single jump: the reconstructed b must not create new extrema of u
    # after one small explicit Euler step (ENO property of WENO + LF split)
    n = 200
    p = _params(n, M=1.1, L=1.0)
    u = np.where(np.arange(n) < n // 2, 1.0, 0.0)[None, :]
    dt = 0.2 * (1.0 / n) / (p.B * 1.1)
    un = u + dt * oracle.weno_rhs(p, u)
    assert un.max() <= 1.0 + 1e-3 and un.min() >= -1e-3


def test_weno_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    for eps in (1e-6, 1e-2):
        for _ in range(5):
            v = rng.standard_normal(5) * 0.3
            g = oracle.weno_grad(v, eps)
            h = 1e-6
            for j in range(5):
                e = np.zeros(5); e[j] = h
                fd = (oracle.weno_parts(v + e, eps)[2] - oracle.weno_parts(v - e, eps)[2]) / (2 * h)
                assert abs(g[j] - fd) < 1e-6 * max(1.0, abs(fd))


def test_weno_transpose_is_adjoint_of_linearisation():
    rng = np.random.default_rng(5)
    p = _params(48, ny=3)
    u = rng.standard_normal((3, 48))
    v = rng.standard_normal((3, 48))
    w = rng.standard_normal((3, 48))
    h = 1e-6
    jv = (oracle.weno_rhs(p, u + h * v) - oracle.weno_rhs(p, u - h * v)) / (2 * h)
    jtw = oracle.weno_rhs_T(p, u, w)
    assert abs(np.sum(jv * w) - np.sum(v * jtw)) < 1e-6 * abs(np.sum(v * jtw))
