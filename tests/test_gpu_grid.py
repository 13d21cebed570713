"""GPU parity of the grouped grid integrator (Brusselator reaction-diffusion,
one coupled system, Newton + left-preconditioned GMRES) against the oracle's
grouped integrator.  The host-side step control takes the oracle's decisions
in FP64 on norms that differ only by reduction order, so the whole run
follows the oracle's step sequence: every counter (steps, right-hand sides,
setups, Newton and GMRES iterations, failures) must equal the oracle's and
the final states agree elementwise to 1e-3 of the error weights (FP64; the
runs measured agree to 4e-8), or 2e-3 with the preconditioner and the GMRES
operator in FP32 (precision 1: each Krylov product carries FP32 rounding, the
runs measured agree to 1.3e-4).  Grids of 6^3, 10^3 and 32^3 (98 304
unknowns: many blocks per reduction and a 3-D launch tiling) and lines of
40 and 200 points."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu


def run_grid(p, tout, rtol, atol, y0=None, maxl=5, device_io=True, precision=0):
    y0 = p.y0 if y0 is None else y0
    with bdfb.Integrator(p, rtol=rtol, atol=atol, maxl=maxl, precision=precision) as I:
        if device_io:
            I.init(0.0, torch.from_numpy(np.ascontiguousarray(y0)).cuda())
            y = torch.empty(y0.size, dtype=torch.float64, device="cuda")
            ret = I.integrate(tout, y)
            y = y.cpu().numpy()
        else:
            I.init(0.0, y0.copy())
            y = np.empty(y0.size)
            ret = I.integrate(tout, y)
        return ret, y, I.cell_stats()[0], I.stats()


MATCH_TOL = {0: 1e-3, 1: 2e-3}


def check_system(y, gs, yo, so, yt, rtol, atol, precision):
    """same step sequence as the oracle: equal counters, elementwise agreement"""
    assert np.array_equal(gs[:8], so[:8]), (gs[:8], so[:8])
    d = np.max(np.abs(y - yo) / (rtol * np.abs(yo) + atol))
    assert d <= MATCH_TOL[precision], d
    w = rtol * np.abs(yt) + atol
    eg, eo = np.max(np.abs(y - yt) / w), np.max(np.abs(yo - yt) / w)
    assert eg <= eo + 10.0 * MATCH_TOL[precision], (eg, eo)
    assert gs[6] > 0                                         # GMRES iterations


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,tout", [(6, 0.05), (10, 0.02), (32, 0.1)])
def test_grid_matches_oracle(nx, tout, precision):
    """precision 1: FP32 preconditioner and GMRES operator"""
    p = gen.brusselator3d(nx, seed=nx)
    rtol, atol = 1e-6, 1e-10
    ret, y, gs, _ = run_grid(p, tout, rtol, atol, precision=precision)
    assert ret == 0
    ro, yo, so = oracle.bruss_integrate(p, 0.0, tout, rtol, atol, maxl=5)
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, tout, 1e-10, 1e-14, maxl=5)
    assert ro == 0 and rt == 0
    check_system(y, gs, yo, so, yt, rtol, atol, precision)


def test_grid_64_matches_oracle():
    """64^3 (786 432 unknowns, 91 steps to t = 0.05): the multi-block reductions
    and the 3-D launch tiling at a size where every kernel runs many blocks per
    SM; in both precisions every counter equals the oracle's and the states
    agree within the match tolerance"""
    p = gen.brusselator3d(64, seed=64)
    rtol, atol, tout = 1e-6, 1e-10, 0.05
    ro, yo, so = oracle.bruss_integrate(p, 0.0, tout, rtol, atol, maxl=5)
    assert ro == 0
    for precision in (0, 1):
        ret, y, gs, _ = run_grid(p, tout, rtol, atol, precision=precision)
        assert ret == 0
        assert np.array_equal(gs[:8], so[:8]), (precision, gs[:8], so[:8])
        d = np.max(np.abs(y - yo) / (rtol * np.abs(yo) + atol))
        assert d <= MATCH_TOL[precision], (precision, d)


def test_grid_steady_state_stays():
    p = gen.brusselator3d(8, noise=0.0)
    ret, y, _, _ = run_grid(p, 0.1, 1e-6, 1e-10)
    assert ret == 0
    assert np.max(np.abs(y - p.y0) / np.abs(p.y0)) <= 1e-12


def test_grid_fourier_mode_decay_and_host_io():
    nx, k = 8, (1, 2, 0)
    npts = nx ** 3
    i, j, l = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    mode = np.cos(2 * np.pi * (k[0] * i + k[1] * j + k[2] * l) / nx).reshape(-1)
    y0 = np.zeros(3 * npts)
    y0[npts:2 * npts] = mode
    p = gen.Brusselator3D(nx=nx, A=0.0, B=0.0, eps=5e-6, D=1e-2, y0=y0)
    lam = -(4.0 * nx * nx) * sum(np.sin(np.pi * kd / nx) ** 2 for kd in k)
    L = p.D * lam
    tout = 0.5 / abs(L)
    ret, y, _, _ = run_grid(p, tout, 1e-8, 1e-12, device_io=False)
    assert ret == 0
    assert np.max(np.abs(y[npts:2 * npts] - np.exp(L * tout) * mode)) <= 20 * 1e-8


def test_grid_64_cubed_properties():
    """A mid-size grid in the benchmark's launch configuration: finite, the
    fast species on its slow manifold w = B / (1 + eps u)."""
    p = gen.brusselator3d(64, seed=3)
    ret, y, gs, st = run_grid(p, 0.05, 1e-6, 1e-10)
    assert ret == 0 and np.all(np.isfinite(y))
    u, v, w = y.reshape(3, -1)
    assert np.max(np.abs(w - p.B / (1.0 + p.eps * u)) / w) < 1e-5
    assert gs[0] > 0 and st["nsteps"] == gs[0]


@pytest.mark.parametrize("precision", [0, 1])
def test_grid_256_cubed_steady_state(precision):
    """The benchmark's 256^3 grid (50 331 648 unknowns) in its launch
    configuration: started at the exact steady state it must stay there."""
    p = gen.brusselator3d(256, noise=0.0)
    ret, y, gs, _ = run_grid(p, 0.1, 1e-6, 1e-10, precision=precision)
    assert ret == 0
    assert np.max(np.abs(y - p.y0) / np.abs(p.y0)) <= 1e-12
    assert gs[0] > 0


# ------------------------------------------------ the 1-D advection demo (Sec. 7)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,length,tout", [(40, 10.0, 0.5), (200, 100.0, 1.0)])
def test_line_matches_oracle(nx, length, tout, precision):
    """The demo problem (paper's initial state) against the oracle's grouped
    integrator, as for the 3-D grid."""
    p = gen.brusselator1d(nx, length=length)
    rtol, atol = 1e-6, 1e-10
    ret, y, gs, _ = run_grid(p, tout, rtol, atol, precision=precision)
    assert ret == 0
    ro, yo, so = oracle.bruss_integrate(p, 0.0, tout, rtol, atol, maxl=5)
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, tout, 1e-10, 1e-14, maxl=5)
    assert ro == 0 and rt == 0
    check_system(y, gs, yo, so, yt, rtol, atol, precision)


def test_line_50k_points_matches_oracle():
    """The demo problem at the benchmark's grid spacing (5e4 points on a line
    of length 5, dx = 1e-4, 125 steps to t = 1): in both precisions every
    counter equals the oracle's and the states agree within the match
    tolerance"""
    p = gen.brusselator1d(50_000, length=5.0)
    rtol, atol, tout = 1e-6, 1e-10, 1.0
    ro, yo, so = oracle.bruss_integrate(p, 0.0, tout, rtol, atol, maxl=5)
    assert ro == 0
    for precision in (0, 1):
        ret, y, gs, _ = run_grid(p, tout, rtol, atol, precision=precision)
        assert ret == 0
        assert np.array_equal(gs[:8], so[:8]), (precision, gs[:8], so[:8])
        d = np.max(np.abs(y - yo) / (rtol * np.abs(yo) + atol))
        assert d <= MATCH_TOL[precision], (precision, d)


def test_line_uniform_steady_state_stays_at_1e6_points():
    nx = 1_000_000
    u, v, w = gen.brusselator_steady_state(1.0, 3.5, 5e-6)
    y0 = np.concatenate([np.full(nx, u), np.full(nx, v), np.full(nx, w)])
    p = gen.Brusselator1D(nx=nx, A=1.0, B=3.5, eps=5e-6, c=0.01, length=1000.0, y0=y0)
    ret, y, gs, _ = run_grid(p, 1.0, 1e-6, 1e-10)
    assert ret == 0
    assert np.max(np.abs(y - y0) / y0) <= 1e-12


@pytest.mark.parametrize("c", [0.01, -0.02])
def test_line_fourier_mode_of_pure_advection(c):
    """v advected alone (u = w = 0, A = B = 0): the exact solution of the
    upwind-discretised system, for either direction of the wind."""
    nx, k, length = 1000, 7, 10.0
    y0 = np.zeros(3 * nx)
    j = np.arange(nx)
    th = 2 * np.pi * k / nx
    y0[nx:2 * nx] = np.cos(th * j)
    p = gen.Brusselator1D(nx=nx, A=0.0, B=0.0, eps=5e-6, c=c, length=length, y0=y0)
    dx = length / nx
    lam1 = -(c / dx) * (1 - np.exp(-1j * th)) if c >= 0 else -(c / dx) * (np.exp(1j * th) - 1)
    tout = 1.0 / abs(lam1)
    ret, y, gs, _ = run_grid(p, tout, 1e-8, 1e-12, device_io=False)
    assert ret == 0
    exact = np.real(np.exp(lam1 * tout) * np.exp(1j * th * j))
    assert np.max(np.abs(y[nx:2 * nx] - exact)) <= 20 * 1e-8


@pytest.mark.parametrize("maxl", [1, 2, 16])
def test_grid_krylov_dimensions(maxl):
    """GMRES(1), GMRES(2) and GMRES(16) against the oracle's GMRES of the same
    dimension (inexact Newton with a short basis, full Krylov with a long one)"""
    p = gen.brusselator3d(6, seed=2)
    ret, y, gs, _ = run_grid(p, 0.05, 1e-6, 1e-10, maxl=maxl)
    assert ret == 0
    ro, yo, so = oracle.bruss_integrate(p, 0.0, 0.05, 1e-6, 1e-10, maxl=maxl)
    rt, yt, _ = oracle.bruss_integrate(p, 0.0, 0.05, 1e-10, 1e-14, maxl=5)
    assert ro == 0 and rt == 0
    check_system(y, gs, yo, so, yt, 1e-6, 1e-10, 0)


def test_grid_op_profile():
    """Option "profile": every vector operation of the step loop is timed with
    events and its algorithmic bytes counted; the run's result is the
    unprofiled one bit for bit, the counted bytes follow the per-kind
    formulas, and the timed operations fit inside the integration's span."""
    p = gen.brusselator3d(32, seed=4)
    N = p.y0.size
    ret0, y0, gs0, st0 = run_grid(p, 0.05, 1e-6, 1e-10)
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, maxl=5) as I:
        I.set_option("profile", 1)
        I.init(0.0, torch.from_numpy(p.y0).cuda())
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        assert I.integrate(0.05, y) == 0
        prof, st = I.op_profile(), I.stats()
    assert ret0 == 0 and np.array_equal(y.cpu().numpy(), y0)
    for k in ("wrms_norm", "dot_prod_multi", "linear_combination", "predict", "accept", "error_weights",
              "newton_update", "rhs", "gmres_operator", "block_setup", "precondition_rhs", "unscale"):
        n, ms, gb = prof[k]
        assert n > 0 and ms > 0 and gb > 0, k
    n, ms, gb = prof["wrms_norm"]
    assert abs(gb - n * 16 * N * 1e-9) <= 1e-9 * gb            # 16 bytes per element
    n, ms, gb = prof["error_weights"]
    assert n >= gs0[0]                                         # one per step at least
    assert abs(gb - n * 24 * N * 1e-9) <= 1e-9 * gb
    assert prof["gmres_operator"][0] == gs0[6]                 # one operator per GMRES iteration
    total_ms = sum(v[1] for v in prof.values())
    assert total_ms <= st["last_kernel_ms"] * 1.01
    with bdfb.Integrator(gen.robertson(4)) as I:
        with pytest.raises(bdfb.BdfbError):
            I.op_profile()                                     # not a grid context
