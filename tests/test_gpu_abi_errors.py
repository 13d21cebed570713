"""Error behaviour of a live context through the C ABI: every rejected call
returns BDFB_ILL_INPUT (nothing traps, nothing is left half-done), and the
context still integrates correctly afterwards -- the result equals that of a
context that never saw the bad calls, bitwise."""
import math

import numpy as np
import pytest
import torch

from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu
L = bdfb.lib
ILL = bdfb.ILL_INPUT


def reference_run(p, tout):
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10) as I:
        I.init(0.0, p.y0.copy())
        y = np.empty(p.y0.size)
        st = np.empty(p.ncell, np.int32)
        assert I.integrate(tout, y, st) == 0
        return y


@pytest.mark.parametrize("kind", ["mass_action", "robertson"])
def test_rejected_calls_leave_the_context_usable(kind):
    p = gen.mass_action(100000, seed=12).subset(np.arange(96)) if kind == "mass_action" else gen.robertson(64)
    tout = 1e-3 if kind == "mass_action" else 40.0
    y_ref = reference_run(p, tout)
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10) as I:
        h = I.h
        y = np.empty(p.y0.size)
        st = np.empty(p.ncell, np.int32)
        yp, sp = y.ctypes.data, st.ctypes.data
        # integrate before init
        assert L.bdfb_integrate(h, tout, yp, sp, bdfb.MEM_HOST) == ILL
        # bad tolerances, options and values
        assert L.bdfb_set_tolerances(h, -1.0, 1e-10) == ILL
        assert L.bdfb_set_tolerances(h, 1e-6, 0.0) == ILL
        assert L.bdfb_set_tolerances(h, math.nan, 1e-10) == ILL
        for key, v in ((b"no_such_option", 1), (b"mxstep", 0), (b"qmax", 6), (b"qmax", 0),
                       (b"interp", 2), (b"lsolver", 3), (b"mapping", 16), (b"graph", 2),
                       (b"autotune", -1), (b"grouped", 5)):
            assert L.bdfb_set_option(h, key, v) == ILL, key
        if kind == "robertson":   # the FP32 path's refinement residual needs mass-action data
            assert L.bdfb_set_option(h, b"precision", 1) == ILL
        assert L.bdfb_set_option(h, b"precision", 2) == ILL
        # bad init arguments
        y0 = p.y0.copy()
        assert L.bdfb_init(h, math.nan, y0.ctypes.data, bdfb.MEM_HOST) == ILL
        assert L.bdfb_init(h, 0.0, None, bdfb.MEM_HOST) == ILL
        assert L.bdfb_init(h, 0.0, y0.ctypes.data, 7) == ILL
        I.init(0.0, y0)
        # bad integrate arguments after a good init
        assert L.bdfb_integrate(h, math.nan, yp, sp, bdfb.MEM_HOST) == ILL
        assert L.bdfb_integrate(h, math.inf, yp, sp, bdfb.MEM_HOST) == ILL
        assert L.bdfb_integrate(h, tout, yp, sp, 7) == ILL
        # the context is intact: the same result as a fresh one, bitwise
        assert L.bdfb_integrate(h, tout, yp, sp, bdfb.MEM_HOST) == 0
        assert np.all(st == 0)
        assert np.array_equal(y, y_ref)


def test_grid_context_rejects_cell_only_options():
    g = gen.brusselator3d(4, seed=3)
    with bdfb.Integrator(g, rtol=1e-6, atol=1e-10) as G:
        h = G.h
        for key, v in ((b"mapping", 32), (b"predictor", 1), (b"lsolver", 1), (b"maxl", 0),
                       (b"maxl", 17), (b"interp", 2)):
            assert L.bdfb_set_option(h, key, v) == ILL, key
        G.init(0.0, torch.from_numpy(g.y0).cuda())
        y = torch.empty(g.y0.size, dtype=torch.float64, device="cuda")
        assert G.integrate(0.01, y) == 0
        assert torch.isfinite(y).all()


def test_shared_network_and_line_reject_foreign_options():
    """a shared-network context takes mxstep, qmax, interp, grouped (0 or 1)
    and lsolver 0 only; the line's own options take 0/1 (device_loop also
    -1); each refusal leaves the context integrating"""
    p = gen.mass_action_banded(32, n=40)
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, shared_network=True) as S:
        for key, v in ((b"mapping", 32), (b"precision", 1), (b"graph", 1), (b"autotune", 1),
                       (b"grouped", 2), (b"predictor", 1), (b"lsolver", 1), (b"interp", 2),
                       (b"qmax", 6), (b"mxstep", 0), (b"mixed_small", 1)):
            assert L.bdfb_set_option(S.h, key, v) == ILL, key
        S.set_option("lsolver", 0)
        S.init(0.0, torch.from_numpy(bdfb.species_major(p)).cuda())
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        assert S.integrate(1e-4, y) == 0
        s0 = np.add.reduceat(p.y0, p.y_off[:-1])
        s1 = np.add.reduceat(bdfb.cell_major(p, y.cpu().numpy()), p.y_off[:-1])
        assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12
    q = gen.brusselator1d(64, length=10.0)
    with bdfb.Integrator(q, rtol=1e-6, atol=1e-10) as Q:
        for key, v in ((b"imex", 2), (b"device_loop", 2), (b"device_loop", -2), (b"precision", 2),
                       (b"maxl", 0), (b"mapping", 32), (b"mixed_small", 1)):
            assert L.bdfb_set_option(Q.h, key, v) == ILL, key
        Q.set_option("imex", 1)
        Q.init(0.0, torch.from_numpy(q.y0).cuda())
        y = torch.empty(q.y0.size, dtype=torch.float64, device="cuda")
        assert Q.integrate(0.1, y) == 0
        assert torch.isfinite(y).all()
