"""Pins of the oracle's IMEX additive Runge-Kutta integrator (the
demonstration problem's integrator, Sec. 7: advection explicit, reaction
implicit; method ARK3(2)4L[2]SA of Kennedy and Carpenter).

* The tables: third-order conditions for the explicit and the implicit
  table with the shared weights, abscissae equal to the row sums, the
  embedded weights of order two (and not three), stiff accuracy, a constant
  ESDIRK diagonal, L-stability and A-stability of the implicit table.
* Fixed steps: observed order three on a linear split problem, on a
  nonlinear split problem with a closed form, and on the exact upwind
  Fourier mode of the advection operator alone.
* Adaptive runs: the demonstration problem against an independent
  tight-tolerance BDF integration, and its uniform steady state.
"""
import numpy as np
import pytest

import oracle
from paper_2011_12984_b300 import gen


def test_tables_order_conditions():
    c, AE, AI, b, bh = oracle.ark_table()
    one = np.ones(4)
    for A in (AE, AI):
        np.testing.assert_allclose(A @ one, c, atol=1e-15)
        assert abs(b @ one - 1) < 1e-15
        assert abs(b @ c - 1 / 2) < 1e-15
        assert abs(b @ (c * c) - 1 / 3) < 1e-15
        assert abs(b @ A @ c - 1 / 6) < 1e-15
    # coupling conditions of order three
    assert abs(b @ AE @ c - 1 / 6) < 1e-15 and abs(b @ AI @ c - 1 / 6) < 1e-15
    assert np.all(np.triu(AE) == 0)                       # explicit
    assert np.all(np.triu(AI, 1) == 0) and AI[0, 0] == 0  # ESDIRK, explicit first stage
    assert np.all(AI[1:, 1:].diagonal() == AI[1, 1])
    np.testing.assert_array_equal(b, AI[3])              # stiffly accurate
    assert abs(bh @ one - 1) < 1e-15 and abs(bh @ c - 1 / 2) < 1e-15
    assert abs(bh @ (c * c) - 1 / 3) > 1e-3               # the embedding is order 2


def stability(A, b, z):
    return 1 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))


def test_implicit_table_l_and_a_stable():
    c, AE, AI, b, bh = oracle.ark_table()
    # L-stable: R(z) ~ C / z as z -> -infinity
    r4, r6 = abs(stability(AI, b, -1e4)), abs(stability(AI, b, -1e6))
    assert r4 < 1e-3 and 90 < r4 / r6 < 110
    for y in np.linspace(0.0, 1e3, 2001):
        assert abs(stability(AI, b, 1j * y)) <= 1 + 1e-12
    # the explicit table is not: |R| grows on the negative real axis
    assert abs(stability(AE, b, -10.0)) > 1


def observed_orders(run, hs):
    errs = np.array([run(h) for h in hs])
    return np.log2(errs[:-1] / errs[1:]), errs


def test_fixed_step_order_linear():
    le, li = -1.0, -2.0
    fe = lambda t, y: le * y
    fi = lambda t, y: li * y
    solve = lambda t, y, g, x: x / (1 - g * li)

    def run(h):
        y, r, st = oracle.ark_integrate(fe, fi, solve, [1.0], 0.0, 1.0, fixed_h=h, rtol=1e-12, atol=1e-14)
        assert r == 0
        return abs(y[0] - np.exp(le + li))
    p, errs = observed_orders(run, [1 / 16, 1 / 32, 1 / 64, 1 / 128])
    assert np.all((p > 2.75) & (p < 3.3)), (p, errs)


def test_fixed_step_order_nonlinear():
    """y' = -y^2 (explicit) - y (implicit): y = 1 / ((1 + 1/y0) e^t - 1)"""
    fe = lambda t, y: -y * y
    fi = lambda t, y: -y
    solve = lambda t, y, g, x: x / (1 + g)
    y0 = 0.8
    exact = 1.0 / ((1 + 1 / y0) * np.exp(1.0) - 1)

    def run(h):
        y, r, st = oracle.ark_integrate(fe, fi, solve, [y0], 0.0, 1.0, fixed_h=h, rtol=1e-12, atol=1e-14)
        assert r == 0
        return abs(y[0] - exact)
    p, errs = observed_orders(run, [1 / 8, 1 / 16, 1 / 32, 1 / 64])
    assert np.all((p > 2.7) & (p < 3.4)), (p, errs)


def test_fixed_step_order_upwind_fourier_mode():
    """Advection alone (explicit part): the semi-discrete solution of
    a' = -c (a_i - a_{i-1}) / dx for a = Re e^{i k x} decays and moves with
    the upwind operator's eigenvalue lam = -(c/dx)(1 - e^{-i k dx})."""
    n, L, c, k = 32, 1.0, 1.0, 2 * np.pi
    dx = L / n
    x = np.arange(n) * dx
    lam = -(c / dx) * (1 - np.exp(-1j * k * dx))
    fe = lambda t, y: -(c / dx) * (y - np.roll(y, 1))
    fi = lambda t, y: np.zeros_like(y)
    solve = lambda t, y, g, xx: xx
    T = 0.25
    exact = np.real(np.exp(1j * k * x) * np.exp(lam * T))

    def run(h):
        y, r, st = oracle.ark_integrate(fe, fi, solve, np.cos(k * x), 0.0, T, fixed_h=h, rtol=1e-12, atol=1e-14)
        assert r == 0
        return np.max(np.abs(y - exact))
    p, errs = observed_orders(run, [T / 16, T / 32, T / 64, T / 128])
    assert np.all((p > 2.8) & (p < 3.3)), (p, errs)


def test_adaptive_linear_within_tolerance():
    fe = lambda t, y: -1.0 * y
    fi = lambda t, y: -50.0 * y
    solve = lambda t, y, g, x: x / (1 + 50.0 * g)
    y, r, st = oracle.ark_integrate(fe, fi, solve, [1.0, 2.0], 0.0, 0.2, rtol=1e-6, atol=1e-12)
    assert r == 0 and st["nst"] > 5
    ex = np.array([1.0, 2.0]) * np.exp(-51.0 * 0.2)
    assert np.max(np.abs(y - ex) / (1e-6 * np.abs(ex) + 1e-12)) <= 10.0


@pytest.mark.parametrize("length", [10.0, 100.0])
def test_demo_against_bdf_truth(length):
    p = gen.brusselator1d(400, length=length)
    r, y, st = oracle.bruss_ark_integrate(p, 0.0, 1.0, 1e-6, 1e-10)
    assert r == 0 and st[0] > 10
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, 1.0, 1e-10, 1e-14)
    assert rt == 0
    w = np.abs(y - yt) / (1e-6 * np.abs(yt) + 1e-10)
    assert w.max() <= 10.0, w.max()
    # Newton: the exact 3x3 Newton converges in about two iterations
    assert st[3] <= 3 * 3 * st[0] + 3 * 3 * st[4]


def test_demo_uniform_steady_state():
    p = gen.brusselator1d(64, length=10.0)
    A, B, eps = p.A, p.B, p.eps
    w = B / (1 + eps * A)
    y0 = np.concatenate([np.full(64, A), np.full(64, w / A), np.full(64, w)])
    r, y, st = oracle.bruss_ark_integrate(p, 0.0, 2.0, 1e-6, 1e-10, y0=y0)
    assert r == 0
    # w's rate (B - w)/eps magnifies the rounding of the stored steady state
    # by 1/eps = 2e5: the fast species settles within ~1e-11 of it
    assert np.max(np.abs(y - y0) / np.abs(y0)) <= 1e-10
