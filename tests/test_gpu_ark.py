"""GPU parity of the IMEX additive Runge-Kutta integrator (option "imex" on
the 1-D demonstration problem, Sec. 7) against the oracle's.

The GPU takes the oracle's decisions up to rounding (the Newton blocks are
inverted by the adjugate formula instead of pivoted LU, the norms are summed
in another order): step and failure counts agree within 3 %, and the final
states differ by a small fraction of the tolerance.  Against a tight BDF
integration the result is within 10 weighted units.  At 10^6 points the
steady state is kept, and without advection every point is an independent
3-species system whose samples are checked against tight single-point
integrations.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-6, 1e-10


def run_imex(p, tout, y0=None, device_io=True, touts=None, precision=0):
    y0 = p.y0 if y0 is None else y0
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, imex=1, precision=precision) as I:
        outs = []
        if device_io:
            I.init(0.0, torch.from_numpy(y0).cuda())
            for t in (touts or [tout]):
                y = torch.empty(y0.size, dtype=torch.float64, device="cuda")
                r = I.integrate(t, y)
                assert r == 0, bdfb.strerror(r)
                outs.append(y.cpu().numpy())
        else:
            I.init(0.0, y0.copy())
            for t in (touts or [tout]):
                y = np.empty(y0.size)
                r = I.integrate(t, y)
                assert r == 0, bdfb.strerror(r)
                outs.append(y)
        return outs, I.cell_stats()[0], I.stats()


def werr(y, yr):
    return np.abs(y - yr) / (RTOL * np.abs(yr) + ATOL)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,length,tout", [(1000, 10.0, 1.0), (20011, 100.0, 0.5), (4096, 1000.0, 3.0)])
def test_against_oracle(nx, length, tout, precision):
    """precision 1 solves the Newton blocks in FP32: the same residual test,
    Newton counts within 10 % instead of 3 %"""
    p = gen.brusselator1d(nx, length=length)
    (y,), cs, st = run_imex(p, tout, precision=precision)
    ro, yo, so = oracle.bruss_ark_integrate(p, 0.0, tout, RTOL, ATOL)
    assert ro == 0
    assert abs(cs[0] - so[0]) <= max(2, 0.03 * so[0]), (cs, so)
    assert abs(cs[5] - so[5]) <= max(1, 0.03 * so[0])
    assert abs(cs[3] - so[3]) <= max(3, (0.03 if precision == 0 else 0.10) * so[3]), (cs, so)
    assert werr(y, yo).max() <= 0.5, werr(y, yo).max()
    if nx <= 4096:
        rt, yt, _ = oracle.bruss_integrate(p, 0.0, tout, 1e-10, 1e-14)
        assert rt == 0
        assert werr(y, yt).max() <= 10.0
    assert st["nsteps"] == cs[0] and st["nniters"] == cs[3]


def test_host_io_and_several_outputs():
    p = gen.brusselator1d(2000, length=10.0)
    outs, cs, _ = run_imex(p, None, device_io=False, touts=[0.25, 0.5, 1.0])
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, 1.0, 1e-10, 1e-14)
    assert werr(outs[-1], yt).max() <= 10.0
    assert np.all(np.isfinite(outs[0])) and not np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", [0, 1])
def test_steady_state_one_million_points(precision):
    p = gen.brusselator1d(1_000_000, length=100.0)
    A, B, eps = p.A, p.B, p.eps
    w = B / (1 + eps * A)
    n = p.nx
    y0 = np.concatenate([np.full(n, A), np.full(n, w / A), np.full(n, w)])
    (y,), cs, _ = run_imex(p, 2.0, y0=y0, precision=precision)
    # precision 0: the rounding equilibrium of the fast species (1/eps = 2e5
    # magnifies the stored state's rounding); precision 1: the FP32 blocks
    # leave each Newton solve at its test, far inside the tolerance (1e-2 rtol)
    assert np.max(np.abs(y - y0) / np.abs(y0)) <= (1e-10 if precision == 0 else 1e-8)
    assert cs[4] == 0 and cs[5] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_no_advection_points_independent(precision):
    """c = 0: each point is its own 3-species ODE; samples against tight
    single-point BDF integrations (rtol 1e-10), and points whose initial
    values are bitwise equal end bitwise equal."""
    nx, length = 1_000_000, 100.0
    p = gen.brusselator1d(nx, length=length, c=0.0)
    (y,), cs, _ = run_imex(p, 1.0, precision=precision)
    idx = np.array([0, 1, 12345, nx // 4, nx // 2 - 1, nx // 2, 777777, nx - 1])
    for q in idx:
        one = gen.brusselator1d(2, length=length, c=0.0)
        y0 = np.array([p.y0[q], p.y0[q], p.y0[nx + q], p.y0[nx + q], p.y0[2 * nx + q], p.y0[2 * nx + q]])
        rt, yt, _ = oracle.bruss_integrate(one, 0.0, 1.0, 1e-10, 1e-14, y0=y0)
        assert rt == 0
        got = np.array([y[q], y[nx + q], y[2 * nx + q]])
        assert werr(got, yt[[0, 2, 4]]).max() <= 10.0, (q, got, yt)
    q = np.arange(1, nx // 2)
    same = np.ones(q.size, bool)
    for s in range(3):
        same &= p.y0[s * nx + q] == p.y0[s * nx + nx - q]
    assert same.sum() > 1000
    for s in range(3):
        np.testing.assert_array_equal(y[s * nx + q[same]], y[s * nx + nx - q[same]])


def test_imex_needs_init_after_option():
    p = gen.brusselator1d(128, length=10.0)
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL) as I:
        I.init(0.0, torch.from_numpy(p.y0).cuda())
        I.set_option("imex", 1)
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        with pytest.raises(bdfb.BdfbError):
            I.integrate(0.1, y)
        I.init(0.0, torch.from_numpy(p.y0).cuda())
        assert I.integrate(0.1, y) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_device_loop_matches_host_loop(precision):
    """The step loop in one cooperative launch (default) takes the host-driven
    loop's decisions: the same method and readings, sums in another order."""
    p = gen.brusselator1d(20011, length=100.0)
    out = {}
    for loop in (0, 1):
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, imex=1, precision=precision, device_loop=loop) as I:
            I.init(0.0, torch.from_numpy(p.y0).cuda())
            y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
            assert I.integrate(0.25, y) == 0
            assert I.integrate(0.5, y) == 0          # a second call continues the state
            out[loop] = (y.cpu().numpy(), I.cell_stats()[0])
    (yh, sh), (yd, sd) = out[0], out[1]
    assert abs(int(sd[0]) - int(sh[0])) <= 2 and abs(int(sd[5]) - int(sh[5])) <= 2, (sd, sh)
    assert werr(yd, yh).max() <= 0.5


@pytest.mark.parametrize("device_loop", [0, 1])
def test_negative_advection_speed(device_loop):
    """c < 0: the upwind difference looks forward; both step loops"""
    p = gen.brusselator1d(1000, length=10.0, c=-0.02)
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, imex=1, device_loop=device_loop) as I:
        I.init(0.0, torch.from_numpy(p.y0).cuda())
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        assert I.integrate(1.0, y) == 0
        cs = I.cell_stats()[0]
    ro, yo, so = oracle.bruss_ark_integrate(p, 0.0, 1.0, RTOL, ATOL)
    assert ro == 0
    assert abs(int(cs[0]) - int(so[0])) <= max(2, 0.03 * so[0])
    assert werr(y.cpu().numpy(), yo).max() <= 0.5
