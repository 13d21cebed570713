"""GPU parity of the per-cell Newton solves by an explicit FP64 inverse
(option "lsolver" 1): at every Jacobian setup each cell's M = I - gamma J is
inverted by Gauss-Jordan elimination with partial pivoting (the block inverse
of the demonstration problem's task-local solver, Sec. 7, for any block
size), and each Newton iteration solves by one product with the inverse.

In exact arithmetic the solves equal the LU ones, so the run takes the
oracle's decisions up to rounding: the cell-by-cell bars of the per-cell
parity tests (cells with the oracle's counters agree with it to 1e-3 of the
error weights; every cell within 3x its oracle error + 10 of an rtol 1e-10
truth; distributions and mean step counts as the oracle's), in every kernel
variant (automatic tiles, one warp per cell, autotuned), on Robertson and
on mass action; linear invariants to rounding; options that cannot combine
with it are refused.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, oracle.host_threads()))


def werr(y, yr, prob, rtol, atol):
    w = np.abs(y - yr) / (rtol * np.abs(yr) + atol)
    return np.maximum.reduceat(w, prob.y_off[:-1])


def run(prob, tout, rtol, atol, **opts):
    with bdfb.Integrator(prob, rtol=rtol, atol=atol, **opts) as I:
        I.init(0.0, torch.from_numpy(prob.y0).cuda())
        y = torch.empty(prob.y0.size, dtype=torch.float64, device="cuda")
        st = torch.empty(prob.ncell, dtype=torch.int32, device="cuda")
        r = I.integrate(tout, y, st)
        torch.cuda.synchronize()
        assert r == 0, bdfb.strerror(r)
        assert np.all(st.cpu().numpy() == 0)
        return y.cpu().numpy(), I.cell_stats(), I.mapping()


def check(p, tout, rtol, atol, y, cs, **bars):
    from test_gpu_cells import check_against_oracle
    check_against_oracle(p, tout, rtol, atol, y, cs, **bars)


@pytest.mark.parametrize("opts", [{}, {"mapping": 32}, {"autotune": 1}, {"graph": 1}])
def test_mass_action_inverse_solves(opts):
    """1536 cells of the mixed-size workload (3/10/32/54 species: every class tiling)"""
    p = gen.mass_action(100000).subset(np.arange(1536))
    y, cs, _ = run(p, 1e-3, 1e-6, 1e-10, lsolver=1, **opts)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0)) <= 5e-11
    check(p, 1e-3, 1e-6, 1e-10, y, cs)


def test_robertson_inverse_solves():
    p = gen.robertson(1000)
    y, cs, _ = run(p, 40.0, 1e-4, 1e-8, lsolver=1)
    assert np.max(np.abs(y.reshape(-1, 3).sum(axis=1) - 1.0)) <= 1e-12
    check(p, 40.0, 1e-4, 1e-8, y, cs)


def test_lu_and_inverse_runs_agree_closely():
    """the same cells with LU and with the inverse: most cells take identical
    step sequences, so their states agree far below the tolerance"""
    p = gen.mass_action(100000, seed=11).subset(np.arange(512))
    y0, c0, _ = run(p, 1e-3, 1e-6, 1e-10)
    y1, c1, _ = run(p, 1e-3, 1e-6, 1e-10, lsolver=1)
    same = c0[:, 0] == c1[:, 0]
    assert same.mean() >= 0.9, same.mean()
    d = werr(y1, y0, p, 1e-6, 1e-10)
    assert np.median(d) <= 0.01, np.median(d)


def test_invalid_combinations_refused():
    p = gen.mass_action(64, seed=1).subset(np.arange(8))
    I = bdfb.Integrator(p)
    try:
        with pytest.raises(RuntimeError):
            I.set_option("lsolver", 2)
        I.set_option("lsolver", 1)
        with pytest.raises(RuntimeError):
            I.set_option("predictor", 1)
        I.set_option("lsolver", 0)
    finally:
        I.close()
    g = gen.brusselator3d(4, seed=1)
    with bdfb.Integrator(g) as G:
        G.set_option("lsolver", 0)
        with pytest.raises(RuntimeError):
            G.set_option("lsolver", 1)


def test_grouped_refuses_inverse_solves():
    p = gen.mass_action(64, seed=1).subset(np.arange(8))
    with bdfb.Integrator(p, grouped=1, lsolver=1) as I:
        I.init(0.0, p.y0.copy())
        y = np.empty(p.y0.size)
        with pytest.raises(bdfb.BdfbError) as e:
            I.integrate(1e-4, y)
        assert e.value.code == bdfb.ILL_INPUT
