"""Pins of the oracle's step-size and order choice after an accepted step.

The reading (the paper is silent; the survey's proposal): candidate ratios
eta_q = 1 / ((6 dsm)^(1/(q+1)) + 1e-6), eta_{q-1} = 1 / ((6 d_{q-1})^(1/q) +
1e-6) for q > 1 and eta_{q+1} = 1 / ((10 d_{q+1})^(1/(q+2)) + 1e-6) for
q < qmax; the largest wins, ties keep q and then prefer q - 1; h changes only
when the winner is at least 1.5; the ratio is capped at 1e4 before the first
increase and at 10 after.  Each case below is built by hand so that one
rule decides it: exact ties use test quantities whose scaled values are
powers of two (6 x and 10 x exact in double, their roots exact), so the
competing ratios are equal bit for bit (checked as a precondition).
"""
import math

import pytest

import oracle

HALF = 1.0 / (0.5 + 1e-6)        # the ratio of a root equal to 1/2
ONE = 1.0 / (1.0 + 1e-6)         # the ratio of a root equal to 1


def exact(target, safety):
    """a double x with safety * x == target exactly (target a power of two)"""
    x = target / safety
    for k in range(-4, 5):
        c = x + k * math.ulp(x)
        if safety * c == target:
            return c
    raise AssertionError("no exact product")


def test_preconditions_of_the_exact_ties():
    assert math.pow(0.25, 1 / 2) == math.pow(0.125, 1 / 3) == math.pow(0.0625, 1 / 4) == 0.5
    assert math.pow(1.0 / 32, 1 / 5) == 0.5


def test_keep_h_below_threshold():
    """every candidate below 1.5: h is kept"""
    changed, q, eta = oracle.bdf_choose(2, exact(1.0, 6), exact(1.0, 6), exact(1.0, 10))
    assert not changed


def test_threshold_1_5():
    """the same order's ratio at 1.49 keeps h, at 1.51 changes it"""
    for target, want in ((1.49, False), (1.51, True)):
        root = 1.0 / target - 1e-6                       # eta_q = target
        dsm = root ** 2 / 6.0                            # q = 1: (6 dsm)^(1/2) = root
        changed, q, eta = oracle.bdf_choose(1, dsm, 0.0, exact(1.0, 10))
        assert changed == want
        if want:
            assert q == 1 and abs(eta - target) <= 1e-12


@pytest.mark.parametrize("q,winner,want_q", [(3, "q-1", 2), (3, "q", 3), (3, "q+1", 4)])
def test_largest_ratio_wins(q, winner, want_q):
    """one candidate's root is 1/2 (ratio ~2), the others' roots 1 (ratio ~1);
    the winner's ratio is exactly HALF only with its own safety factor (6, 6
    and 10) and root order (q + 1, q, q + 2)"""
    dsm, dqm1, dqp1 = exact(1.0, 6), exact(1.0, 6), exact(1.0, 10)
    if winner == "q":
        dsm = exact(0.5 ** (q + 1), 6)
    elif winner == "q-1":
        dqm1 = exact(0.5 ** q, 6)
    else:
        dqp1 = exact(0.5 ** (q + 2), 10)
    changed, qn, eta = oracle.bdf_choose(q, dsm, dqm1, dqp1)
    assert changed and qn == want_q and eta == HALF


def test_tie_q_and_q_plus_1_keeps_q():
    changed, q, eta = oracle.bdf_choose(1, exact(0.25, 6), 0.0, exact(0.125, 10))
    assert changed and q == 1 and eta == HALF


def test_tie_q_and_q_minus_1_keeps_q():
    changed, q, eta = oracle.bdf_choose(2, exact(0.125, 6), exact(0.25, 6), exact(1.0, 10))
    assert changed and q == 2 and eta == HALF


def test_tie_q_minus_1_and_q_plus_1_prefers_q_minus_1():
    changed, q, eta = oracle.bdf_choose(2, exact(1.0, 6), exact(0.25, 6), exact(0.0625, 10))
    assert changed and q == 1 and eta == HALF


@pytest.mark.parametrize("grown,cap", [(False, 1e4), (True, 10.0)])
def test_caps(grown, cap):
    """a tiny error allows eta ~ 1e6: capped at 1e4 before the first
    increase, at 10 after"""
    changed, q, eta = oracle.bdf_choose(2, 1e-30, exact(1.0, 6), exact(1.0, 10), grown_once=grown)
    assert changed and q == 2 and eta == cap


def test_orders_at_the_ends():
    """q = 1 has no lower order (d_{q-1} ignored); q = qmax no higher one"""
    changed, q, eta = oracle.bdf_choose(1, exact(1.0, 6), 1e-30, exact(1.0, 10))
    assert not changed
    changed, q, eta = oracle.bdf_choose(5, exact(1.0, 6), exact(1.0, 6), 1e-30, qmax=5)
    assert not changed
    changed, q, eta = oracle.bdf_choose(3, exact(1.0, 6), exact(1.0, 6), 1e-30, qmax=3)
    assert not changed
