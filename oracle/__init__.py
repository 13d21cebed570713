"""CPU oracle for the batched BDF/Newton hot path.

TEST INFRASTRUCTURE ONLY.  This package may be imported only by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  The library under ``paper_2011_12984_b300`` never
imports it, and it never imports that library: the two share no code; only
the seeded input generators (``paper_2011_12984_b300.gen``, which contain no
method arithmetic) feed both.

The arithmetic lives in plain C (``oracle/*.c``: IEEE double, no FMA
contraction), loaded here through ctypes.  ctypes releases the GIL during a
foreign call, so independent cells can be integrated on several host threads.
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_lib = None

_d = C.c_double
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)
_pi32 = C.POINTER(C.c_int32)
_pi64 = C.POINTER(C.c_int64)
_pu8 = C.POINTER(C.c_uint8)
_pi = C.POINTER(C.c_int)

SUCCESS, TOO_MUCH_WORK, ERR_FAILURE, CONV_FAILURE = 0, -1, -3, -4
QMAX = 5


class Options(C.Structure):
    _fields_ = [("rtol", _d), ("atol", _d), ("mxstep", _i64), ("qmax", C.c_int),
                ("fixed_h", _d), ("fixed_q", C.c_int), ("h0", _d),
                ("trace_y", _pd), ("trace_acor", _pd), ("trace_cap", _i64), ("z_init", _pd),
                ("interp", C.c_int)]


class Cells(C.Structure):
    _fields_ = [("kind", C.c_int), ("ncell", _i64), ("n", _pi32), ("y_off", _pi64),
                ("rxn_off", _pi64), ("reac", _pu8), ("prod", _pu8), ("k", _pd)]


class Bruss(C.Structure):
    _fields_ = [("nx", C.c_int), ("A", _d), ("B", _d), ("eps", _d), ("D", _d), ("dim", C.c_int),
                ("c", _d), ("len", _d)]


_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, _d, _pd, _pd)
_SOLVE = C.CFUNCTYPE(C.c_int, C.c_void_p, _d, _pd, _d, _pd)


class ImexSystem(C.Structure):
    _fields_ = [("N", _i64), ("user", C.c_void_p), ("fe", _FN), ("fi", _FN), ("isolve", _SOLVE)]


class ArkOptions(C.Structure):
    _fields_ = [("rtol", _d), ("atol", _d), ("mxstep", _i64), ("fixed_h", _d)]


class ArkStats(C.Structure):
    _fields_ = [("nst", _i64), ("nfe", _i64), ("nfi", _i64), ("nni", _i64), ("ncfn", _i64),
                ("netf", _i64), ("hlast", _d), ("tcur", _d)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.or_wrms_norm.restype = _d
        L.or_linear_integrate.argtypes = [_i64, _pd, C.c_int, _pd, _d, _pd, _d,
                                          C.POINTER(Options), _pd, _pi64, _pi64]
        L.or_cells_integrate.argtypes = [C.POINTER(Cells), _i64, _i64, _d, _pd, _d, _d, _d,
                                         _i64, _pd, _pi32, _pi64]
        L.or_cells_integrate_mode.argtypes = [C.POINTER(Cells), _i64, _i64, _d, _pd, _d, _d, _d,
                                              _i64, C.c_int, _pd, _pi32, _pi64]
        L.or_cells_integrate_grouped.argtypes = [C.POINTER(Cells), _d, _pd, _d, _d, _d, _i64,
                                                 C.c_int, _pd, _pi64]
        L.or_ark_table.argtypes = [_pd, _pd, _pd, _pd, _pd]
        L.or_ark_integrate.argtypes = [C.POINTER(ImexSystem), C.POINTER(ArkOptions), _d, _pd, _d,
                                       _pd, C.POINTER(ArkStats)]
        L.or_bruss_ark_integrate.argtypes = [C.POINTER(Bruss), _d, _pd, _d, _d, _d, _i64, _pd, _pi64]
        L.or_bruss_gmres.argtypes = [C.POINTER(Bruss), _pd, _d, _pd, _d, C.c_int, _pd, _pd]
        L.or_bruss_integrate.argtypes = [C.POINTER(Bruss), _d, _pd, _d, _d, _d, C.c_int, _i64,
                                         C.c_int, _pd, _pi64]
        _lib = L
    return _lib


def _p(a, t=_pd):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptrs(vs):
    return (_pd * len(vs))(*[_p(v) for v in vs])


# ---------------------------------------------------------------- vectors
def scale(c, x):
    x = _f64(x)
    z = np.empty_like(x)
    lib().or_scale(_i64(x.size), _d(c), _p(x), _p(z))
    return z


def const(c, n):
    z = np.empty(n)
    lib().or_const(_i64(n), _d(c), _p(z))
    return z


def abs_(x):
    x = _f64(x)
    z = np.empty_like(x)
    lib().or_abs(_i64(x.size), _p(x), _p(z))
    return z


def inv(x):
    x = _f64(x)
    z = np.empty_like(x)
    lib().or_inv(_i64(x.size), _p(x), _p(z))
    return z


def add_const(x, b):
    x = _f64(x)
    z = np.empty_like(x)
    lib().or_add_const(_i64(x.size), _p(x), _d(b), _p(z))
    return z


def error_weights(rtol, atol, y):
    y = _f64(y)
    w = np.empty_like(y)
    lib().or_error_weights(_i64(y.size), _d(rtol), _d(atol), _p(y), _p(w))
    return w


def linear_sum(a, x, b, y):
    x, y = _f64(x), _f64(y)
    z = np.empty_like(x)
    lib().or_linear_sum(_i64(x.size), _d(a), _p(x), _d(b), _p(y), _p(z))
    return z


def linear_combination(c, xs):
    xs = [_f64(x) for x in xs]
    c = _f64(c)
    z = np.empty_like(xs[0])
    lib().or_linear_combination(_i64(z.size), C.c_int(len(xs)), _p(c), _ptrs(xs), _p(z))
    return z


def scale_add_multi(a, x, ys):
    x = _f64(x)
    ys = [_f64(y) for y in ys]
    a = _f64(a)
    zs = [np.empty_like(x) for _ in ys]
    lib().or_scale_add_multi(_i64(x.size), C.c_int(len(ys)), _p(a), _p(x), _ptrs(ys), _ptrs(zs))
    return zs


def dot_prod_multi(x, ys):
    """returns (d, sum |x_i y_ji|) per j"""
    x = _f64(x)
    ys = [_f64(y) for y in ys]
    d = np.empty(len(ys))
    s = np.empty(len(ys))
    lib().or_dot_prod_multi(_i64(x.size), C.c_int(len(ys)), _p(x), _ptrs(ys), _p(d), _p(s))
    return d, s


def wrms_norm(x, w):
    x, w = _f64(x), _f64(w)
    return lib().or_wrms_norm(_i64(x.size), _p(x), _p(w))


# ---------------------------------------------------------------- dense LU
def lu_factor(A):
    A = _f64(A).copy()
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    info = lib().or_lu_factor(C.c_int(n), _p(A), _p(piv, _pi))
    return A, piv, info


def lu_solve(lu, piv, b):
    b = _f64(b).copy()
    lib().or_lu_solve(C.c_int(lu.shape[0]), _p(lu), _p(piv, _pi), _p(b))
    return b


# ---------------------------------------------------------------- BDF core
def bdf_constants(q):
    """(l[0..q], E_q, E_{q-1}, E_{q+1})"""
    l = np.zeros(QMAX + 2)
    out = np.zeros(3)
    lib().or_bdf_constants(C.c_int(q), _p(l), _p(out))
    return l[:q + 1], out[0], out[1], out[2]


def bdf_choose(q, dsm, dqm1=0.0, dqp1=0.0, qmax=QMAX, grown_once=False):
    """the step-size/order choice after an accepted step: (changed, q_new, eta)"""
    L = lib()
    L.or_bdf_choose.argtypes = [C.c_int, C.c_int, C.c_int, _d, _d, _d, _pi, _pd]
    qn, eta = C.c_int(q), _d(1.0)
    r = L.or_bdf_choose(q, qmax, int(grown_once), dsm, dqm1, dqp1, C.byref(qn), C.byref(eta))
    return bool(r), qn.value, eta.value


def linear_integrate(A, Cs, t0, y0, tout, rtol=1e-6, atol=1e-10, fixed_h=0.0, fixed_q=0,
                     h0=0.0, mxstep=100000, trace=0, z_init=None, interp=False):
    """y' = A y + sum_k Cs[k] t^k.  Returns (ret, y, stats, trace_y, trace_acor)."""
    A = _f64(np.atleast_2d(A))
    N = A.shape[0]
    Cs = _f64(np.zeros((1, N)) if Cs is None or len(Cs) == 0 else np.atleast_2d(Cs))
    y0 = _f64(y0)
    y = np.empty(N)
    st = np.zeros(8, dtype=np.int64)
    ty = np.zeros((max(trace, 1), N))
    ta = np.zeros((max(trace, 1), N))
    zi = None if z_init is None else _f64(z_init)
    opt = Options(rtol, atol, mxstep, QMAX, fixed_h, fixed_q, h0,
                  _p(ty) if trace else None, _p(ta) if trace else None, trace,
                  None if zi is None else _p(zi), int(interp))
    nt = _i64(0)
    ret = lib().or_linear_integrate(N, _p(A), Cs.shape[0], _p(Cs), t0, _p(y0), tout,
                                    C.byref(opt), _p(y), _p(st, _pi64), C.byref(nt))
    return ret, y, st, ty[:nt.value], ta[:nt.value]


# ---------------------------------------------------------------- problems
def robertson_rhs(k, y):
    k, y = _f64(k), _f64(y)
    f = np.empty(3)
    lib().or_robertson_rhs(_p(k), _p(y), _p(f))
    return f


def robertson_jac(k, y):
    k, y = _f64(k), _f64(y)
    J = np.empty((3, 3))
    lib().or_robertson_jac(_p(k), _p(y), _p(J))
    return J


def massaction_rhs(reac, prod, k, y):
    reac = np.ascontiguousarray(reac, np.uint8)
    prod = np.ascontiguousarray(prod, np.uint8)
    k, y = _f64(k), _f64(y)
    f = np.empty(y.size)
    lib().or_massaction_rhs(C.c_int(y.size), C.c_int(k.size), _p(reac, _pu8), _p(prod, _pu8),
                            _p(k), _p(y), _p(f))
    return f


def massaction_jac(reac, prod, k, y):
    reac = np.ascontiguousarray(reac, np.uint8)
    prod = np.ascontiguousarray(prod, np.uint8)
    k, y = _f64(k), _f64(y)
    n = y.size
    J = np.empty((n, n))
    lib().or_massaction_jac(C.c_int(n), C.c_int(k.size), _p(reac, _pu8), _p(prod, _pu8),
                            _p(k), _p(y), _p(J))
    return J


def _cells_struct(prob):
    """ctypes view of a generator problem; the arrays stay alive in ``keep``."""
    if prob.kind == "robertson":
        n = np.ascontiguousarray(prob.n, np.int32)
        y_off = np.ascontiguousarray(prob.y_off, np.int64)
        k = _f64(prob.k)
        keep = (n, y_off, k)
        s = Cells(0, prob.ncell, _p(n, _pi32), _p(y_off, _pi64), None, None, None, _p(k))
    else:
        n = np.ascontiguousarray(prob.n, np.int32)
        y_off = np.ascontiguousarray(prob.y_off, np.int64)
        rxn_off = np.ascontiguousarray(prob.rxn_off, np.int64)
        reac = np.ascontiguousarray(prob.reactants, np.uint8)
        prod = np.ascontiguousarray(prob.products, np.uint8)
        k = _f64(prob.k)
        keep = (n, y_off, rxn_off, reac, prod, k)
        s = Cells(1, prob.ncell, _p(n, _pi32), _p(y_off, _pi64), _p(rxn_off, _pi64),
                  _p(reac, _pu8), _p(prod, _pu8), _p(k))
    return s, keep


def integrate_cells(prob, t0, tout, rtol, atol, mxstep=100000, cells=None, threads=1,
                    y0=None, interp=False):
    """Integrate the listed cells (default all) independently; returns
    (y, status, stats[ncell, 8]) over the whole problem (cells not listed keep y0
    and status 1).  ``threads`` > 1 spreads cell ranges over host threads."""
    s, keep = _cells_struct(prob)
    y0 = _f64(prob.y0 if y0 is None else y0)
    y = y0.copy()
    status = np.full(prob.ncell, 1, np.int32)
    stats = np.zeros((prob.ncell, 8), np.int64)
    L = lib()
    if cells is None:
        nch = max(1, threads * 8) if threads > 1 else 1
        b = np.linspace(0, prob.ncell, nch + 1).astype(np.int64)
        ranges = [(int(b[i]), int(b[i + 1])) for i in range(nch) if b[i + 1] > b[i]]
    else:
        cells = np.sort(np.asarray(cells, dtype=np.int64))
        ranges = [(int(c), int(c) + 1) for c in cells]

    def run(r):
        return L.or_cells_integrate_mode(C.byref(s), r[0], r[1], t0, _p(y0), tout, rtol, atol, mxstep,
                                         int(interp), _p(y), _p(status, _pi32), _p(stats, _pi64))

    if threads <= 1:
        for r in ranges:
            run(r)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, ranges))
    del keep
    return y, status, stats


def integrate_cells_grouped(prob, t0, tout, rtol, atol, mxstep=100000, y0=None, interp=False):
    """All cells as one system with task-local Newton solves (one step size and
    order, error test over every species); returns (y, ret, stats[8])."""
    s, keep = _cells_struct(prob)
    y0 = _f64(prob.y0 if y0 is None else y0)
    y = y0.copy()
    stats = np.zeros(8, np.int64)
    ret = lib().or_cells_integrate_grouped(C.byref(s), t0, _p(y0), tout, rtol, atol, mxstep,
                                           int(interp), _p(y), _p(stats, _pi64))
    del keep
    return y, ret, stats


def bruss_struct(p):
    """the 3-D reaction-diffusion grid, or the 1-D advection line (p.kind ==
    "brusselator1d": speed p.c on [0, p.length))"""
    if getattr(p, "kind", "") == "brusselator1d":
        return Bruss(p.nx, p.A, p.B, p.eps, 0.0, 1, p.c, p.length)
    return Bruss(p.nx, p.A, p.B, p.eps, p.D, 3, 0.0, 1.0)


def bruss_rhs(p, y):
    s = bruss_struct(p)
    y = _f64(y)
    f = np.empty_like(y)
    lib().or_bruss_rhs(C.byref(s), _p(y), _p(f))
    return f


def bruss_jv(p, y, v):
    s = bruss_struct(p)
    y, v = _f64(y), _f64(v)
    jv = np.empty_like(y)
    lib().or_bruss_jv(C.byref(s), _p(y), _p(v), _p(jv))
    return jv


def bruss_gmres(p, y, gamma, ewt, tol, maxl, b):
    s = bruss_struct(p)
    y, ewt = _f64(y), _f64(ewt)
    x = _f64(b).copy()
    rn = _d(0)
    it = lib().or_bruss_gmres(C.byref(s), _p(y), gamma, _p(ewt), tol, maxl, _p(x), C.byref(rn))
    return x, it, rn.value


def bruss_integrate(p, t0, tout, rtol, atol, maxl=5, mxstep=100000, y0=None, interp=False):
    s = bruss_struct(p)
    y0 = _f64(p.y0 if y0 is None else y0)
    y = np.empty_like(y0)
    st = np.zeros(8, np.int64)
    ret = lib().or_bruss_integrate(C.byref(s), t0, _p(y0), tout, rtol, atol, maxl, mxstep,
                                   int(interp), _p(y), _p(st, _pi64))
    return ret, y, st


# ---------------------------------------------------------------- IMEX ARK
def ark_table():
    """the ARK3(2)4L[2]SA tables as the oracle holds them: (c, AE, AI, b, bhat)"""
    c, b, bh = np.zeros(4), np.zeros(4), np.zeros(4)
    AE, AI = np.zeros((4, 4)), np.zeros((4, 4))
    lib().or_ark_table(_p(c), _p(AE), _p(AI), _p(b), _p(bh))
    return c, AE, AI, b, bh


def ark_integrate(fe, fi, isolve, y0, t0, tout, rtol=1e-6, atol=1e-10, fixed_h=0.0, mxstep=100000):
    """The oracle's IMEX ARK on Python callbacks (small systems only):
    fe(t, y) and fi(t, y) return arrays; isolve(t, y, gamma, x) returns
    (I - gamma J_I(t, y))^{-1} x.  Returns (y, ret, stats dict)."""
    y0 = _f64(y0)
    N = y0.size

    def wrap(fun):
        def cb(user, t, y, f):
            out = fun(t, np.ctypeslib.as_array(y, (N,)).copy())
            np.ctypeslib.as_array(f, (N,))[:] = out
            return 0 if np.all(np.isfinite(out)) else 1
        return _FN(cb)

    def cbs(user, t, y, g, x):
        xv = np.ctypeslib.as_array(x, (N,))
        xv[:] = isolve(t, np.ctypeslib.as_array(y, (N,)).copy(), g, xv.copy())
        return 0

    cfe, cfi, csolve = wrap(fe), wrap(fi), _SOLVE(cbs)
    sys_ = ImexSystem(N, None, cfe, cfi, csolve)
    opt = ArkOptions(rtol, atol, mxstep, fixed_h)
    st = ArkStats()
    y = np.empty(N)
    ret = lib().or_ark_integrate(C.byref(sys_), C.byref(opt), t0, _p(y0), tout, _p(y), C.byref(st))
    stats = {k: getattr(st, k) for k, _ in ArkStats._fields_}
    return y, ret, stats


def bruss_ark_integrate(p, t0, tout, rtol, atol, mxstep=100000, y0=None):
    """the 1-D demonstration problem by IMEX ARK (advection explicit, reaction
    implicit); returns (ret, y, stats[8] = nst, nfe, nfi, nni, ncfn, netf)"""
    s = bruss_struct(p)
    y0 = _f64(p.y0 if y0 is None else y0)
    y = np.empty_like(y0)
    st = np.zeros(8, np.int64)
    ret = lib().or_bruss_ark_integrate(C.byref(s), t0, _p(y0), tout, rtol, atol, mxstep, _p(y),
                                       _p(st, _pi64))
    return ret, y, st


# ---------------------------------------------------------------- MLP
MLP_NPARAM = 5642


def mlp_forward(params, X, bf16=False):
    """network outputs; bf16: with the BF16 operands of the tensor-core form
    (weights, inputs and hidden activations rounded, exact accumulation)"""
    params, X = _f64(params), _f64(np.atleast_2d(X))
    Y = np.empty((X.shape[0], 10))
    fn = lib().or_mlp_forward_bf16 if bf16 else lib().or_mlp_forward
    fn(_p(params), _i64(X.shape[0]), _p(X), _p(Y))
    return Y


def mlp_loss_grad(params, X, T, bf16=False):
    """(loss, gradient); bf16: back-propagation with BF16 operands"""
    params, X, T = _f64(params), _f64(np.atleast_2d(X)), _f64(np.atleast_2d(T))
    g = np.empty(MLP_NPARAM)
    L = lib()
    fn = L.or_mlp_loss_grad_bf16 if bf16 else L.or_mlp_loss_grad
    fn.restype = _d
    loss = fn(_p(params), _i64(X.shape[0]), _p(X), _p(T), _p(g))
    return loss, g


def bf16_round(x):
    """elementwise round to nearest bfloat16 (ties to even)"""
    L = lib()
    L.or_bf16_round.restype = _d
    L.or_bf16_round.argtypes = [_d]
    return np.array([L.or_bf16_round(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def adam_step(params, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """in place on float64 arrays"""
    L = lib()
    L.or_adam_step.argtypes = [_i64, _pd, _pd, _pd, _pd, _i64, _d, _d, _d, _d]
    L.or_adam_step(params.size, _p(params), _p(_f64(g)), _p(m), _p(v), t, lr, b1, b2, eps)


def host_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
