"""Pins of the oracle's Brusselator systems (the 3-D reaction-diffusion grid
and the 1-D advection-reaction demo of Sec. 7) and GMRES.

* the reaction steady state u* = A, w* = B/(1 + eps A), v* = w*/A stays put;
* with u = w = 0 and A = B = 0 the v field diffuses freely: a single Fourier
  mode is an eigenvector of the periodic 7-point Laplacian with eigenvalue
  -(4/dx^2) sum_d sin^2(pi k_d / n), so f, J v and the integrated decay
  exp(D lambda t) are known in closed form;
* J v agrees with central differences of f;
* GMRES with as many Krylov vectors as unknowns equals the dense solve;
* 1-D demo: the paper's initial state, a uniform steady state stays put
  (upwind differences of a constant vanish), a Fourier mode of v under pure
  advection follows the exact solution of the upwind-discretised system for
  either sign of c, J v and full-Krylov GMRES as above.
"""
import numpy as np
import pytest

import oracle
from paper_2011_12984_b300 import gen


def mode(nx, k):
    i, j, l = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    return np.cos(2 * np.pi * (k[0] * i + k[1] * j + k[2] * l) / nx).reshape(-1)


def lam(nx, k):
    dx = 1.0 / nx
    return -(4.0 / dx ** 2) * sum(np.sin(np.pi * kd / nx) ** 2 for kd in k)


def test_steady_state_stays():
    p = gen.brusselator3d(8, noise=0.0)
    ret, y, st = oracle.bruss_integrate(p, 0.0, 0.1, 1e-6, 1e-10)
    assert ret == 0
    # f(y*) is not exactly zero in floating point: (B - w*)/eps cancels to ~1e-10
    assert np.max(np.abs(y - p.y0) / np.abs(p.y0)) <= 1e-12


@pytest.mark.parametrize("interp", [False, True])
def test_fourier_mode_of_free_diffusion(interp):
    """the closed-form decay, in both output modes of the grid integrator"""
    nx, k = 8, (1, 2, 0)
    npts = nx ** 3
    y0 = np.zeros(3 * npts)
    p = gen.Brusselator3D(nx=nx, A=0.0, B=0.0, eps=5e-6, D=1e-2, y0=y0)
    y0[npts:2 * npts] = mode(nx, k)
    f = oracle.bruss_rhs(p, y0)
    L = p.D * lam(nx, k)
    assert np.max(np.abs(f[npts:2 * npts] - L * y0[npts:2 * npts])) <= 1e-10 * abs(L)
    assert np.max(np.abs(f[:npts])) == 0.0 and np.max(np.abs(f[2 * npts:])) == 0.0
    jv = oracle.bruss_jv(p, y0, y0)
    assert np.max(np.abs(jv[npts:2 * npts] - L * y0[npts:2 * npts])) <= 1e-10 * abs(L)
    tout = 0.5 / abs(L)
    ret, y, st = oracle.bruss_integrate(p, 0.0, tout, 1e-8, 1e-12, y0=y0, interp=interp)
    assert ret == 0
    assert np.max(np.abs(y[npts:2 * npts] - np.exp(L * tout) * y0[npts:2 * npts])) <= 20 * 1e-8


def test_jv_matches_difference_quotient():
    p = gen.brusselator3d(4, noise=0.05, seed=4)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(p.y0.size)
    h = 1e-6
    fd = (oracle.bruss_rhs(p, p.y0 + h * v) - oracle.bruss_rhs(p, p.y0 - h * v)) / (2 * h)
    jv = oracle.bruss_jv(p, p.y0, v)
    assert np.max(np.abs(jv - fd)) <= 1e-6 * np.max(np.abs(jv))


def test_gmres_full_krylov_equals_dense_solve():
    p = gen.brusselator3d(2, noise=0.05, seed=8)       # 24 unknowns
    y = p.y0
    N = y.size
    gamma = 2e-5
    J = np.column_stack([oracle.bruss_jv(p, y, e) for e in np.eye(N)])
    M = np.eye(N) - gamma * J
    rng = np.random.default_rng(3)
    b = rng.standard_normal(N)
    ewt = 1.0 / (1e-6 * np.abs(y) + 1e-10)
    x, it, rn = oracle.bruss_gmres(p, y, gamma, ewt, 0.0, N, b)
    xd = np.linalg.solve(M, b)
    assert np.max(np.abs(x - xd)) <= 1e-9 * np.max(np.abs(xd))


def test_gmres_short_krylov_reduces_residual():
    p = gen.brusselator3d(6, noise=0.05, seed=8)
    y = p.y0
    gamma = 1e-3
    rng = np.random.default_rng(4)
    b = rng.standard_normal(y.size) * 1e-6
    ewt = 1.0 / (1e-6 * np.abs(y) + 1e-10)
    x, it, rn = oracle.bruss_gmres(p, y, gamma, ewt, 1e-30, 5, b)
    assert it == 5
    r = b - (x - gamma * oracle.bruss_jv(p, y, x))
    assert np.linalg.norm(r * ewt) < 0.5 * np.linalg.norm(b * ewt)


def test_fast_species_reaches_its_slow_manifold():
    """w relaxes on the 1/eps time scale to w = B/(1 + eps u) (its reaction
    equilibrium for the current u); u and v evolve slowly (B = 3 > 1 + A^2
    makes the homogeneous u-v state oscillatory, so they do not settle)."""
    p = gen.brusselator3d(6, seed=2)
    ret, y, st = oracle.bruss_integrate(p, 0.0, 0.1, 1e-6, 1e-10)
    assert ret == 0
    u, v, w = y.reshape(3, -1)
    assert np.max(np.abs(w - p.B / (1.0 + p.eps * u)) / w) < 1e-6
    w0 = p.y0.reshape(3, -1)[2]
    assert np.max(np.abs(w0 - p.B / (1.0 + p.eps * p.y0.reshape(3, -1)[0])) / w0) > 1e-3
    assert st[6] > 0        # GMRES iterations were used


# ------------------------------------------------ the 1-D advection demo (Sec. 7)
def advect_mode(nx, k, c, length, t):
    """exact solution of the upwind-discretised advection v' = -c D v on the
    periodic line for v(0) = cos(theta j): Re(exp(lambda t) exp(i theta j))
    with theta = 2 pi k / nx and lambda = -(c/dx)(1 - e^{-i theta}) for
    c >= 0 (backward difference), -(c/dx)(e^{i theta} - 1) for c < 0"""
    dx = length / nx
    th = 2 * np.pi * k / nx
    lam1 = -(c / dx) * (1 - np.exp(-1j * th)) if c >= 0 else -(c / dx) * (np.exp(1j * th) - 1)
    j = np.arange(nx)
    return np.real(np.exp(lam1 * t) * np.exp(1j * th * j)), lam1


def test_1d_demo_initial_state():
    p = gen.brusselator1d(40, length=10.0)
    x = np.arange(40) * 0.25
    bump = 0.1 * np.exp(-((x - 5.0) ** 2) / (2 * 2.5 ** 2))
    assert np.allclose(p.y0[:40], 1.0 + bump, rtol=0, atol=1e-15)
    assert np.allclose(p.y0[40:80], 3.5 + bump, rtol=0, atol=1e-15)
    assert np.allclose(p.y0[80:], 3.0 + bump, rtol=0, atol=1e-15)


def test_1d_uniform_steady_state_stays():
    nx = 64
    u, v, w = gen.brusselator_steady_state(1.0, 3.5, 5e-6)
    y0 = np.concatenate([np.full(nx, u), np.full(nx, v), np.full(nx, w)])
    p = gen.Brusselator1D(nx=nx, A=1.0, B=3.5, eps=5e-6, c=0.01, length=10.0, y0=y0)
    f = oracle.bruss_rhs(p, y0)
    assert np.max(np.abs(f[:2 * nx])) <= 1e-13          # advection of a uniform field is exactly 0
    ret, y, st = oracle.bruss_integrate(p, 0.0, 1.0, 1e-6, 1e-10)
    assert ret == 0 and np.max(np.abs(y - y0) / y0) <= 1e-12


def test_1d_fourier_mode_of_pure_advection():
    for c in (0.01, -0.02):
        nx, k, length = 32, 3, 10.0
        y0 = np.zeros(3 * nx)
        y0[nx:2 * nx] = np.cos(2 * np.pi * k * np.arange(nx) / nx)
        p = gen.Brusselator1D(nx=nx, A=0.0, B=0.0, eps=5e-6, c=c, length=length, y0=y0)
        f = oracle.bruss_rhs(p, y0)
        dvdt, lam1 = advect_mode(nx, k, c, length, 0.0)
        exact_f = np.real(lam1 * np.exp(2j * np.pi * k * np.arange(nx) / nx))
        assert np.max(np.abs(f[nx:2 * nx] - exact_f)) <= 1e-13 * abs(lam1)
        assert np.max(np.abs(f[:nx])) == 0.0 and np.max(np.abs(f[2 * nx:])) == 0.0
        tout = 1.0 / abs(lam1)
        ret, y, st = oracle.bruss_integrate(p, 0.0, tout, 1e-8, 1e-12, y0=y0)
        assert ret == 0
        exact, _ = advect_mode(nx, k, c, length, tout)
        assert np.max(np.abs(y[nx:2 * nx] - exact)) <= 20 * 1e-8


def test_1d_jv_and_full_krylov_gmres():
    p = gen.brusselator1d(10, length=10.0)             # 30 unknowns
    rng = np.random.default_rng(5)
    v = rng.standard_normal(p.y0.size)
    h = 1e-6
    fd = (oracle.bruss_rhs(p, p.y0 + h * v) - oracle.bruss_rhs(p, p.y0 - h * v)) / (2 * h)
    jv = oracle.bruss_jv(p, p.y0, v)
    assert np.max(np.abs(jv - fd)) <= 1e-6 * np.max(np.abs(jv))
    N = p.y0.size
    gamma = 2e-5
    J = np.column_stack([oracle.bruss_jv(p, p.y0, e) for e in np.eye(N)])
    M = np.eye(N) - gamma * J
    b = rng.standard_normal(N)
    x, it, rn = oracle.bruss_gmres(p, p.y0, gamma, np.ones(N), 0.0, N, b)
    assert np.max(np.abs(M @ x - b)) <= 1e-10 * np.max(np.abs(b))
