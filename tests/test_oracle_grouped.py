"""Pins of the oracle's grouped integration (all cells as one system with
task-local Newton solves: the grouping of Sec. 2, the demonstration
problem's task-local nonlinear solver of Sec. 7).

* One cell: the task-local Newton iteration on a single block is the global
  Newton iteration, so the grouped run reproduces the per-cell run.
* C identical copies of one cell: the WRMS norm over all C n species equals
  the norm over one copy, and every block iterates exactly like the single
  cell, so the grouped run takes the single cell's steps and C times its
  Newton iterations.  A block norm taken over all N entries instead of the
  block's own n, or a shared rate, breaks this.
* Linear invariants (sum y per mass-action cell, sum y = 1 for Robertson)
  survive the block-wise solves.
* Accuracy against a tight-tolerance truth.
"""
import numpy as np
import pytest

import oracle
from paper_2011_12984_b300 import gen

pytestmark = pytest.mark.filterwarnings("ignore")


def replicate(p, cell, copies):
    return p.subset(np.full(copies, cell, np.int64))


@pytest.mark.parametrize("interp", [False, True])
@pytest.mark.parametrize("kind", ["robertson", "mass_action"])
def test_one_cell_equals_per_cell(kind, interp):
    """in both output modes (the grouped entry point passes the mode through)"""
    p = gen.robertson(5).subset([2]) if kind == "robertson" else gen.mass_action(16, seed=5).subset([7])
    tout = 40.0 if kind == "robertson" else 1e-3
    yg, r, sg = oracle.integrate_cells_grouped(p, 0.0, tout, 1e-6, 1e-10, interp=interp)
    yc, sc, stc = oracle.integrate_cells(p, 0.0, tout, 1e-6, 1e-10, interp=interp)
    assert r == 0 and sc[0] == 0
    assert sg[0] == stc[0, 0] and sg[3] == stc[0, 3] and sg[5] == stc[0, 5]
    np.testing.assert_allclose(yg, yc, rtol=1e-13, atol=1e-20)
    if interp:
        yk, _, _ = oracle.integrate_cells_grouped(p, 0.0, tout, 1e-6, 1e-10)
        assert not np.array_equal(yg, yk)


@pytest.mark.parametrize("copies", [2, 7])
def test_identical_copies_step_like_one_cell(copies):
    base = gen.mass_action(64, seed=9)
    cell = int(np.nonzero(base.n == 10)[0][0])
    one = base.subset([cell])
    many = replicate(base, cell, copies)
    y1, r1, s1 = oracle.integrate_cells_grouped(one, 0.0, 1e-3, 1e-6, 1e-10)
    yc, rc, sc = oracle.integrate_cells_grouped(many, 0.0, 1e-3, 1e-6, 1e-10)
    assert r1 == 0 and rc == 0
    assert sc[0] == s1[0] and sc[5] == s1[5] and sc[4] == s1[4]
    assert sc[3] == copies * s1[3]
    np.testing.assert_allclose(yc.reshape(copies, -1), np.tile(y1, (copies, 1)), rtol=1e-12, atol=1e-20)


def test_invariants_and_accuracy_mass_action():
    p = gen.mass_action(96, seed=3)
    y, r, st = oracle.integrate_cells_grouped(p, 0.0, 1e-3, 1e-6, 1e-10)
    assert r == 0
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12
    yt, stt, _ = oracle.integrate_cells(p, 0.0, 1e-3, 1e-10, 1e-14)
    assert np.all(stt == 0)
    w = np.abs(y - yt) / (1e-6 * np.abs(yt) + 1e-10)
    assert w.max() <= 10.0
    # every cell takes every step: at least as many as the hardest cell alone
    _, _, sc = oracle.integrate_cells(p, 0.0, 1e-3, 1e-6, 1e-10)
    assert st[0] >= 0.5 * sc[:, 0].max()
    assert st[3] >= p.ncell * st[0]      # at least one iteration per cell per step


def test_invariants_and_accuracy_robertson():
    p = gen.robertson(300)
    y, r, st = oracle.integrate_cells_grouped(p, 0.0, 40.0, 1e-4, 1e-8)
    assert r == 0
    assert np.max(np.abs(y.reshape(-1, 3).sum(axis=1) - 1.0)) <= 1e-12
    yt, _, _ = oracle.integrate_cells(p, 0.0, 40.0, 1e-10, 1e-14)
    w = np.abs(y - yt) / (1e-4 * np.abs(yt) + 1e-8)
    assert w.max() <= 10.0


def test_empty_problem():
    p = gen.mass_action(8, seed=1).subset(np.zeros(0, np.int64))
    y, r, st = oracle.integrate_cells_grouped(p, 0.0, 1e-3, 1e-6, 1e-10)
    assert r == 0 and y.size == 0 and st[0] == 0
