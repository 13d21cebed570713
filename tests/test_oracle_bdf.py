"""Pins of the oracle's BDF core against what the mathematics fixes.

* constant-step runs reproduce the textbook BDF_q recurrences (table in
  tests/golden, itself re-derived here from the interpolation definition);
* the local-error constants E_q, E_{q-1}, E_{q+1} turn the quantities the
  integrator monitors into the textbook one-step error of orders q, q-1, q+1;
* adaptive runs meet closed forms of y' = lambda y and y' = A y;
* fixed-step runs converge with order q.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bdf_constant_step.txt")


def load_table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        q, b0, al, c = [s.strip() for s in line.split("|")]
        rows[int(q)] = (Fraction(b0), [Fraction(a) for a in al.split()], Fraction(c))
    return rows


def bdf_from_definition(q):
    """alpha, beta0 of BDF_q from its definition: the degree-q polynomial through
    y_n, ..., y_{n-q} at t = 0, -1, ..., -q has slope f_n at t = 0 (h = 1)."""
    pts = [Fraction(-i) for i in range(q + 1)]
    d = []   # derivative at 0 of the Lagrange basis polynomials
    for i, ti in enumerate(pts):
        s = Fraction(0)
        for m, tm in enumerate(pts):
            if m == i:
                continue
            prod = Fraction(1, 1) / (ti - tm)
            for j, tj in enumerate(pts):
                if j not in (i, m):
                    prod *= (0 - tj) / (ti - tj)
            s += prod
        d.append(s)
    beta0 = 1 / d[0]      # sum d_i y_{n-i} = f_n, normalised to alpha_0 = 1
    return beta0, [di / d[0] for di in d]


def test_golden_table_matches_definition():
    tab = load_table()
    for q in range(1, 6):
        b0, al = bdf_from_definition(q)
        assert b0 == tab[q][0]
        assert al == tab[q][1]
        # error constant: plug y = t^{q+1}/(q+1)! (y^{(q+1)} = 1) into the formula
        fq = Fraction(1)
        for i in range(2, q + 2):
            fq *= i
        tau = sum(a * Fraction(-i) ** (q + 1) for i, a in enumerate(al)) / fq
        assert abs(tau) == tab[q][2]


def test_coefficients_l():
    # l_1 = 1/beta_0 of the textbook formula; l_q = 1/q!
    tab = load_table()
    for q in range(1, 6):
        l, Eq, _, _ = oracle.bdf_constants(q)
        assert l[0] == 1.0
        assert abs(l[1] - float(1 / tab[q][0])) < 1e-15
        assert abs(l[q] - 1.0 / np.prod(np.arange(1, q + 1))) < 1e-16


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_constant_step_run_is_textbook_bdf(q):
    """After q steps at constant h the Nordsieck corrector makes y_n satisfy the
    textbook BDF_q recurrence exactly (to rounding) on a linear system."""
    tab = load_table()
    b0, al, _ = tab[q]
    A = np.array([[-1.0, 0.5], [0.2, -3.0]])
    h = 0.02
    ret, y, st, ty, ta = oracle.linear_integrate(A, None, 0.0, [1.0, -0.5], 40 * h,
                                                 fixed_h=h, fixed_q=q, trace=60)
    assert ret == 0 and len(ty) == 40
    Y = np.vstack([[1.0, -0.5], ty])
    for n in range(q + 1, len(Y)):
        lhs = sum(float(al[i]) * Y[n - i] for i in range(q + 1))
        rhs = h * float(b0) * (A @ Y[n])
        assert np.max(np.abs(lhs - rhs)) < 1e-14, (q, n, lhs - rhs)


def poly_run(q, deg, h, nsteps):
    """fixed-step order-q run on y' = deg t^(deg-1), y(0) = 0 (y = t^deg)"""
    Cs = np.zeros((deg, 1))
    Cs[deg - 1, 0] = deg
    ret, y, st, ty, ta = oracle.linear_integrate([[0.0]], Cs, 0.0, [0.0], h * nsteps,
                                                 fixed_h=h, fixed_q=q, trace=nsteps + 5)
    assert ret == 0
    return ty[:, 0], ta[:, 0]


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_error_constant_Eq(q):
    """E_q * Delta_n equals |C_{q+1}| h^{q+1} y^{(q+1)} (textbook one-step error)."""
    tab = load_table()
    h, n = 0.05, 200
    _, acor = poly_run(q, q + 1, h, n)
    _, Eq, _, _ = oracle.bdf_constants(q)
    D = float(np.prod(np.arange(1, q + 2)))      # y^{(q+1)} of t^{q+1}
    want = float(tab[q][2]) * D * h ** (q + 1)
    # rounding of y ~ (n h)^{q+1} against Delta ~ h^{q+1} limits this to ~1e-5
    assert abs(Eq * acor[-1] - want) <= 1e-4 * want


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_error_constant_Eqm1(q):
    """E_{q-1} * z_q estimates the order-(q-1) one-step error: on y = t^q the
    order-q history has z_q = h^q, and the order-(q-1) error is
    |C_q| h^q y^(q) with y^(q) = q!."""
    tab = load_table()
    h = 0.05
    _, _, Eqm1, _ = oracle.bdf_constants(q)
    want = float(tab[q - 1][2]) * float(np.prod(np.arange(1, q + 1))) * h ** q
    assert abs(Eqm1 * h ** q - want) <= 1e-12 * want


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_error_constant_Eqp1(q):
    """E_{q+1} * (Delta_n - Delta_{n-1}) from an order-q run on y = t^{q+2}
    equals the textbook order-(q+1) one-step error |C_{q+2}| h^{q+2} y^(q+2)."""
    tab = load_table()
    h, n = 0.05, 300
    _, acor = poly_run(q, q + 2, h, n)
    _, _, _, Eqp1 = oracle.bdf_constants(q)
    D = float(np.prod(np.arange(1, q + 3)))
    want = float(tab[q + 1][2]) * D * h ** (q + 2)
    got = Eqp1 * (acor[-1] - acor[-2])
    assert abs(got - want) <= 1e-4 * want


@pytest.mark.parametrize("lam,tout", [(-1.0, 5.0), (-1.0e3, 5.0e-3), (-1.0e6, 5.0e-6)])
def test_scalar_decay_closed_form(lam, tout):
    for rtol in (1e-6, 1e-9):
        ret, y, st, _, _ = oracle.linear_integrate([[lam]], None, 0.0, [1.0], tout,
                                                   rtol=rtol, atol=1e-14)
        exact = np.exp(lam * tout)
        assert ret == 0
        # errors committed while |y| ~ 1 persist as y decays: scale by max |y| = 1
        assert abs(y[0] - exact) <= 20 * rtol + 1e-13
        assert st[6] >= 2          # the order controller left order 1


def test_linear_system_eigen_closed_form():
    """y' = A y with A = V diag(-1, -1e4) V^{-1}: y(t) = V exp(Lt) V^{-1} y0."""
    V = np.array([[1.0, 1.0], [1.0, -2.0]])
    L = np.array([-1.0, -1.0e4])
    A = V @ np.diag(L) @ np.linalg.inv(V)
    y0 = np.array([2.0, -1.0])
    for tout in (0.01, 1.0, 3.0):
        ret, y, st, _, _ = oracle.linear_integrate(A, None, 0.0, y0, tout, rtol=1e-8, atol=1e-12)
        exact = V @ (np.exp(L * tout) * np.linalg.solve(V, y0))
        assert ret == 0
        assert np.max(np.abs(y - exact) / (1e-8 * np.abs(exact) + 1e-12)) < 20


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_observed_order(q):
    """global error at t = 1 of fixed-step order-q runs on y' = -y + cos t scales
    like h^q (slope within +-0.15 on a log-log fit)."""
    def err(h):
        n = int(round(1.0 / h))
        # y' = -y + sum c_k t^k with the Taylor polynomial of cos to degree 20
        # (truncation 1/22! ~ 1e-21 at t = 1, below rounding)
        Cs = np.zeros((21, 1))
        for k in range(0, 21, 2):
            Cs[k, 0] = (-1) ** (k // 2) / float(np.prod(np.arange(1, k + 1)))
        # solution y = (cos t + sin t)/2; start from its exact Taylor history
        # z_j = h^j y^(j)(0)/j!, y^(j)(0) = 1/2, 1/2, -1/2, -1/2, ...
        dj = [0.5, 0.5, -0.5, -0.5, 0.5, 0.5]
        zi = np.array([[h ** j * dj[j] / float(np.prod(np.arange(1, j + 1)))] for j in range(q + 1)])
        ret, y, _, _, _ = oracle.linear_integrate([[-1.0]], Cs, 0.0, [0.5], n * h,
                                                  fixed_h=h, fixed_q=q, z_init=zi)
        assert ret == 0
        return abs(y[0] - 0.5 * (np.cos(n * h) + np.sin(n * h)))
    hs = np.array([1 / 40, 1 / 80, 1 / 160, 1 / 320]) if q <= 3 else np.array([1 / 10, 1 / 20, 1 / 40, 1 / 80])
    e = np.array([err(h) for h in hs])
    slope = np.polyfit(np.log(hs), np.log(e), 1)[0]
    assert abs(slope - q) < 0.15, (q, slope, e)


# ---------------------------------------------------------------- output by interpolation
def test_interpolation_exact_for_polynomials():
    """Fixed steps of BDF3 from the exact history on y' = 3 t^2 (y = 1 + t^3):
    the method and the degree-3 history polynomial are exact, so the value at
    a tout off the step grid (s = (tout - t_n)/h in (0, 1/2), a short
    extrapolation, and after a second call, behind the last step) is the cubic
    to rounding.  A wrong sign of s or a wrong power fails it."""
    h, q = 0.1, 3
    t0 = 0.0
    # Nordsieck history of y = 1 + t^3 at t0: z_j = h^j y^(j)(t0) / j!
    z = np.array([[1.0], [0.0], [0.0], [h ** 3]])
    Cs = np.array([[0.0], [0.0], [3.0]])
    for tout in (0.73, 1.04):
        ret, y, st, _, _ = oracle.linear_integrate([[0.0]], Cs, t0, [1.0], tout, fixed_h=h, fixed_q=q,
                                                   z_init=z, interp=True, rtol=1e-12, atol=1e-14)
        assert ret == 0
        assert abs(y[0] - (1.0 + tout ** 3)) <= 1e-12, (tout, y[0])


@pytest.mark.parametrize("lam,tout", [(-1.0, 5.0), (-1.0e3, 5.0e-3)])
def test_interpolated_output_closed_form(lam, tout):
    """Stepping past tout and interpolating meets the same bar as landing on
    tout, with no more steps."""
    for rtol in (1e-6, 1e-9):
        ri, yi, si, _, _ = oracle.linear_integrate([[lam]], None, 0.0, [1.0], tout, rtol=rtol, atol=1e-14,
                                                   interp=True)
        rc, yc, sc, _, _ = oracle.linear_integrate([[lam]], None, 0.0, [1.0], tout, rtol=rtol, atol=1e-14)
        assert ri == 0 and rc == 0
        assert abs(yi[0] - np.exp(lam * tout)) <= 20 * rtol + 1e-13
        assert si[0] <= sc[0]
