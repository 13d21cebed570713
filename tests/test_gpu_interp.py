"""GPU parity of the interpolated output mode (option "interp"): the integrator
steps past tout and returns the history polynomial sum_j z_j s^j at
s = (tout - t_n)/h instead of shortening its last step to land on tout (the
normal output mode of the variable-order BDF integrator, Sec. 3).

Every integrator that runs BDF takes it: independent cells (every size class,
FP64 and mixed precision, graph replay), the grouped system, cells sharing a
sparse network, the 3-D grid and the 1-D line.  Each is compared with the
oracle in the same output mode, with the bars of that integrator's parity tests
(independent cells: the cell-by-cell tiers of the per-cell tests; the systems:
final states against an rtol 1e-10 truth in units of the run's own error
weights, step counts against the oracle's).  Properties that hold exactly:
linear invariants survive the interpolation to rounding; asking twice for the
same tout (no step between) returns the same vector bitwise; a run with
interpolated output differs from the clamped one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen
from test_gpu_cells import check_against_oracle

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, oracle.host_threads()))


def werr_cells(y, yr, prob, rtol, atol):
    w = np.abs(y - yr) / (rtol * np.abs(yr) + atol)
    return np.maximum.reduceat(w, prob.y_off[:-1])


def rms(e):
    return float(np.sqrt(np.mean(e * e)))


def run(prob, touts, rtol, atol, shared=False, **opts):
    """integrate through the listed output times; returns the outputs,
    statuses, per-cell statistics and totals"""
    with bdfb.Integrator(prob, rtol=rtol, atol=atol, shared_network=shared, **opts) as I:
        y0 = bdfb.species_major(prob) if shared else prob.y0
        I.init(0.0, torch.from_numpy(np.ascontiguousarray(y0)).cuda())
        outs = []
        for t in touts:
            y = torch.empty(y0.size, dtype=torch.float64, device="cuda")
            st = torch.empty(max(getattr(prob, "ncell", 1), 1), dtype=torch.int32, device="cuda")
            r = I.integrate(t, y, st)
            torch.cuda.synchronize()
            assert r == 0, bdfb.strerror(r)
            yv = y.cpu().numpy()
            outs.append(bdfb.cell_major(prob, yv) if shared else yv)
        return outs, I.cell_stats(), I.stats()


@pytest.mark.parametrize("opts", [{}, {"mapping": 32}, {"precision": 1}, {"graph": 1},
                                  {"autotune": 1}])
def test_cells_interp_matches_oracle(opts):
    """1536 cells of the mixed-size mass-action workload (3/10/32/54 species)"""
    p = gen.mass_action(100000).subset(np.arange(1536))
    rtol, atol, tout = 1e-6, 1e-10, 1e-3
    (y,), cs, _ = run(p, [tout], rtol, atol, interp=1, **opts)
    check_against_oracle(p, tout, rtol, atol, y, cs, interp=True)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0)) <= 5e-11                      # conservation survives


def test_cells_interp_robertson():
    p = gen.robertson(1000)
    (y,), cs, _ = run(p, [40.0], 1e-4, 1e-8, interp=1)
    assert np.max(np.abs(y.reshape(-1, 3).sum(axis=1) - 1.0)) <= 1e-12
    check_against_oracle(p, 40.0, 1e-4, 1e-8, y, cs, min_seq=0.9, min_same=1.0, interp=True)


def test_cells_interp_sequence_and_repeat():
    """outputs at 2.5e-4, 5e-4, 5e-4 again and 1e-3: each within the bar of a
    single run to that time; the repeated request (no step between) returns
    the same vector bitwise; the clamped mode gives a different final vector"""
    p = gen.mass_action(100000, seed=6).subset(np.arange(256))
    rtol, atol = 1e-6, 1e-10
    touts = [2.5e-4, 5e-4, 5e-4, 1e-3]
    outs, cs, _ = run(p, touts, rtol, atol, interp=1)
    assert np.array_equal(outs[1], outs[2])
    for t, y in zip(touts, outs):
        yo, _, _ = oracle.integrate_cells(p, 0.0, t, rtol, atol, threads=THREADS, interp=True)
        yt, _, _ = oracle.integrate_cells(p, 0.0, t, 1e-10, 1e-14, threads=THREADS)
        eg, eo = werr_cells(y, yt, p, rtol, atol), werr_cells(yo, yt, p, rtol, atol)
        assert np.all(eg <= max(10.0, 2.0 * eo.max())), (t, eg.max(), eo.max())
    (yc,), _, _ = run(p, [1e-3], rtol, atol)
    assert not np.array_equal(yc, outs[-1])


def test_grouped_interp_matches_oracle():
    p = gen.mass_action(100000, seed=2).subset(np.arange(256))
    rtol, atol, tout = 1e-6, 1e-10, 1e-3
    (y,), _, stats = run(p, [tout], rtol, atol, grouped=1, interp=1)
    yt, _, _ = oracle.integrate_cells(p, 0.0, tout, 1e-10, 1e-14, threads=THREADS)
    w = lambda v: np.abs(v - yt) / (rtol * np.abs(yt) + atol)
    # one grouped run is one trajectory: oracle runs at rtol (1 + k 1e-12),
    # k = -5..5, part by rounding alone and span RMS errors 0.5-2.0 here
    worst_max = worst_rms = 0.0
    nst = []
    for k in range(-5, 6):
        yo, ro, s = oracle.integrate_cells_grouped(p, 0.0, tout, rtol * (1.0 + k * 1e-12), atol, interp=True)
        assert ro == 0
        nst.append(s[0])
        worst_max, worst_rms = max(worst_max, w(yo).max()), max(worst_rms, rms(w(yo)))
    eg = w(y)
    assert eg.max() <= max(10.0, 2.0 * worst_max), (eg.max(), worst_max)
    assert rms(eg) <= max(0.05, 1.5 * worst_rms), (rms(eg), worst_rms)
    assert 0.95 * min(nst) <= stats["nsteps"] // p.ncell <= 1.05 * max(nst)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12


def test_shared_network_interp():
    """cells sharing one banded 128-species network: against the oracle's
    grouped integration in the same output mode (dense LU per cell)"""
    p = gen.mass_action_banded(96, n=128)
    rtol, atol, tout = 1e-6, 1e-10, 1e-3
    (y,), _, stats = run(p, [tout], rtol, atol, shared=True, interp=1)
    yt, _, _ = oracle.integrate_cells(p, 0.0, tout, 1e-10, 1e-14, threads=THREADS)
    w = lambda v: np.abs(v - yt) / (rtol * np.abs(yt) + atol)
    worst_max = worst_rms = 0.0
    for f in (1.0, 1.0 + 1e-12, 1.0 - 1e-12):
        yo, ro, _ = oracle.integrate_cells_grouped(p, 0.0, tout, rtol * f, atol, interp=True)
        assert ro == 0
        worst_max, worst_rms = max(worst_max, w(yo).max()), max(worst_rms, rms(w(yo)))
    eg = w(y)
    assert eg.max() <= max(10.0, 2.0 * worst_max), (eg.max(), worst_max)
    assert rms(eg) <= max(0.05, 1.5 * worst_rms), (rms(eg), worst_rms)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12


@pytest.mark.parametrize("which", ["grid6", "line"])
def test_grid_and_line_interp_match_oracle(which):
    if which == "grid6":
        p, tout = gen.brusselator3d(6, seed=6), 0.05
    else:
        p, tout = gen.brusselator1d(200, length=100.0), 1.0
    rtol, atol = 1e-6, 1e-10
    outs, gs, _ = run(p, [tout, tout], rtol, atol, interp=1)
    y = outs[0]
    assert np.array_equal(outs[0], outs[1])
    ro, yo, so = oracle.bruss_integrate(p, 0.0, tout, rtol, atol, maxl=5, interp=True)
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, tout, 1e-10, 1e-14, maxl=5)
    assert ro == 0 and rt == 0
    wt = rtol * np.abs(yt) + atol
    eg, eo = np.max(np.abs(y - yt) / wt), np.max(np.abs(yo - yt) / wt)
    assert eg <= max(10.0, 1.5 * eo), (eg, eo)
    assert abs(gs[0, 0] / so[0] - 1.0) <= 0.1, (gs[0], so)
    (yc,), _, _ = run(p, [tout], rtol, atol)
    assert not np.array_equal(yc, y)


def test_interp_edge_cases():
    """tout = t0 returns the initial state bitwise (no step, nothing to
    interpolate); a cell stopped by mxstep reports its status and the state
    it reached (t_n < tout: no interpolation), like the clamped mode"""
    p = gen.mass_action(100000, seed=8).subset(np.arange(64))
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, interp=1) as I:
        I.init(0.0, p.y0.copy())
        y = np.empty(p.y0.size)
        st = np.empty(p.ncell, np.int32)
        assert I.integrate(0.0, y, st) == 0
        assert np.array_equal(y, p.y0)
    outs = []
    for interp in (0, 1):
        with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, interp=interp, mxstep=1) as I:
            I.init(0.0, p.y0.copy())
            y = np.empty(p.y0.size)
            st = np.empty(p.ncell, np.int32)
            r = I.integrate(1e-3, y, st)
            assert r == bdfb.TOO_MUCH_WORK and np.all(st == bdfb.TOO_MUCH_WORK)
            outs.append(y.copy())
    # one step from the same start (the first step is at most a tenth of
    # tout - t0, so no clamp applies) is the same in both modes
    assert np.array_equal(outs[0], outs[1])
    assert not np.array_equal(outs[0], p.y0)
