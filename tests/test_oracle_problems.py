"""Pins of the oracle's right-hand sides, Jacobians and per-cell integration.

* Robertson and mass-action RHS against a stoichiometric-matrix formulation
  (S . rates, built independently with numpy), and their conservation law
  1^T f = 0; Jacobians against central differences of the RHS;
* closed forms of mass-action reactions (A -> B first order, A + B -> C + D
  second order with equal initial amounts);
* Robertson cells conserve sum y = 1 to 1e-12 over [0, 40]; mass-action cells
  conserve sum y;
* tiny mass-action cells (n = 3) at tight tolerance agree with scipy's Radau
  integrator (an independent implicit Runge-Kutta code).
"""
import numpy as np
import pytest

import oracle
from paper_2011_12984_b300 import gen


def robertson_by_reactions(k, y):
    # R1: y1 -> y2 (k1 y1); R2: 2 y2 -> y2 + y3 (k2 y2^2); R3: y2 + y3 -> y1 + y3 (k3 y2 y3)
    S = np.array([[-1.0, 0.0, 1.0], [1.0, -1.0, -1.0], [0.0, 1.0, 0.0]])
    rates = np.array([k[0] * y[0], k[1] * y[1] ** 2, k[2] * y[1] * y[2]])
    return S @ rates


def massaction_by_matrix(n, reac, prod, k, y, absolute=False):
    R = np.zeros((n, len(k)))
    P = np.zeros((n, len(k)))
    for r in range(len(k)):
        for s in reac[r]:
            if s != 255:
                R[s, r] += 1
        for s in prod[r]:
            if s != 255:
                P[s, r] += 1
    rates = k * np.prod(np.where(R > 0, y[:, None] ** R, 1.0), axis=0)
    if absolute:                    # sum of |terms| per species (rounding scale)
        return (P + R) @ np.abs(rates)
    return (P - R) @ rates


def fd_jac(f, y, h=1e-7):
    n = y.size
    J = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h * max(abs(y[j]), 1e-2)
        J[:, j] = (f(y + e) - f(y - e)) / (2 * e[j])
    return J


def test_robertson_rhs_and_jacobian():
    rng = np.random.default_rng(1)
    p = gen.robertson(20)
    for c in range(20):
        y = rng.uniform(0.0, 1.0, 3) * np.array([1.0, 1e-4, 1.0])
        k = p.k[c]
        f = oracle.robertson_rhs(k, y)
        ref = robertson_by_reactions(k, y)
        assert np.allclose(f, ref, rtol=1e-14, atol=1e-14 * np.max(np.abs(ref)))
        assert abs(f.sum()) <= 1e-15 * np.sum(np.abs(f)) + 1e-300
        J = oracle.robertson_jac(k, y)
        Jfd = fd_jac(lambda v: oracle.robertson_rhs(k, v), y)
        assert np.max(np.abs(J - Jfd)) <= 1e-6 * np.max(np.abs(J))
        assert np.all(np.abs(J.sum(axis=0)) <= 1e-12 * np.max(np.abs(J)))


def test_massaction_rhs_and_jacobian():
    p = gen.mass_action(40, seed=3)
    rng = np.random.default_rng(2)
    for c in range(40):
        n = int(p.n[c])
        r0, r1 = p.rxn_off[c], p.rxn_off[c + 1]
        reac, prod, k = p.reactants[r0:r1], p.products[r0:r1], p.k[r0:r1]
        y = rng.uniform(0.05, 1.0, n)
        f = oracle.massaction_rhs(reac, prod, k, y)
        ref = massaction_by_matrix(n, reac, prod, k, y)
        scale = massaction_by_matrix(n, reac, prod, k, y, absolute=True)
        assert np.all(np.abs(f - ref) <= 1e-14 * scale)
        assert abs(f.sum()) <= 1e-14 * np.sum(scale)
        J = oracle.massaction_jac(reac, prod, k, y)
        Jfd = fd_jac(lambda v: oracle.massaction_rhs(reac, prod, k, v), y)
        # large opposite rates cancel in f: scale by the derivative of sum |terms|
        Jabs = fd_jac(lambda v: massaction_by_matrix(n, reac, prod, k, v, absolute=True), y)
        assert np.max(np.abs(J - Jfd)) <= 1e-6 * np.max(np.abs(Jabs))
        assert np.max(np.abs(J.sum(axis=0))) <= 1e-13 * np.max(np.abs(Jabs))


def single_problem(n, reac, prod, k, y0):
    R = len(k)
    return gen.MassActionProblem(
        n=np.array([n], np.int32), y_off=np.array([0, n], np.int64),
        rxn_off=np.array([0, R], np.int64),
        reactants=np.array(reac, np.uint8).reshape(R, 4),
        products=np.array(prod, np.uint8).reshape(R, 4),
        k=np.array(k, float), y0=np.array(y0, float))


def test_first_order_reaction_closed_form():
    kr = 3.0
    p = single_problem(2, [[0, 255, 255, 255]], [[1, 255, 255, 255]], [kr], [1.0, 0.0])
    for tout in (0.1, 1.0, 4.0):
        y, st, _ = oracle.integrate_cells(p, 0.0, tout, 1e-9, 1e-14)
        assert st[0] == 0
        ex = np.exp(-kr * tout)
        assert abs(y[0] - ex) <= 20 * 1e-9
        assert abs(y[0] + y[1] - 1.0) <= 1e-13


def test_second_order_reaction_closed_form():
    # A + B -> C + D with A0 = B0: A(t) = A0 / (1 + k A0 t)
    kr, a0 = 50.0, 0.4
    p = single_problem(4, [[0, 1, 255, 255]], [[2, 3, 255, 255]], [kr], [a0, a0, 0.1, 0.1])
    for tout in (0.01, 0.5, 10.0):
        y, st, _ = oracle.integrate_cells(p, 0.0, tout, 1e-9, 1e-14)
        assert st[0] == 0
        ex = a0 / (1.0 + kr * a0 * tout)
        assert abs(y[0] - ex) <= 20 * 1e-9 * a0
        assert abs(y.sum() - 1.0) <= 1e-13


def test_robertson_conserves_mass_all_cells():
    p = gen.robertson(1000)
    y, st, stats = oracle.integrate_cells(p, 0.0, 40.0, 1e-4, 1e-8, threads=4)
    assert np.all(st == 0)
    assert np.max(np.abs(y.reshape(-1, 3).sum(axis=1) - 1.0)) <= 1e-12
    assert np.all(stats[:, 0] > 10)


def test_massaction_conserves_mass():
    p = gen.mass_action(64, seed=5).subset(np.arange(64))
    y, st, stats = oracle.integrate_cells(p, 0.0, 1e-3, 1e-6, 1e-10, threads=4)
    assert np.all(st == 0)
    for c in range(p.ncell):
        s0 = p.y0[p.y_off[c]:p.y_off[c + 1]].sum()
        s1 = y[p.y_off[c]:p.y_off[c + 1]].sum()
        assert abs(s1 - s0) <= 1e-12


def test_tiny_cells_match_independent_radau():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    p = gen.mass_action(200, sizes=(3,), seed=9).subset(np.arange(5))
    y, st, _ = oracle.integrate_cells(p, 0.0, 1e-3, 1e-10, 1e-14)
    assert np.all(st == 0)
    for c in range(p.ncell):
        r0, r1 = p.rxn_off[c], p.rxn_off[c + 1]
        reac, prod, k = p.reactants[r0:r1], p.products[r0:r1], p.k[r0:r1]
        y0 = p.y0[p.y_off[c]:p.y_off[c + 1]]
        f = lambda t, v: massaction_by_matrix(3, reac, prod, k, v)
        sol = scipy_integrate.solve_ivp(f, (0.0, 1e-3), y0, method="Radau", rtol=1e-12,
                                        atol=1e-16)
        yr = sol.y[:, -1]
        yc = y[p.y_off[c]:p.y_off[c + 1]]
        w = 1e-8 * np.abs(yr) + 1e-12
        assert np.max(np.abs(yc - yr) / w) < 10, (c, yc, yr)
