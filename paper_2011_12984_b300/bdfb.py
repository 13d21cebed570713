"""Thin Python binding of ``libbdfb`` (C ABI in ``include/bdfb.h``).

Argument marshalling only: every numerical step runs in the CUDA library.
Device arrays are passed as ``torch.Tensor`` (CUDA, contiguous) and host
arrays as numpy arrays or CPU tensors; the stream defaults to torch's current
stream.  If the shared library is missing this module raises at import time
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BDFB_LIBRARY=phases loads the profiling build with the step-phase timers
# (python -m paper_2011_12984_b300.build --phases)
LIB_PATH = os.path.join(_HERE, "libbdfb_phases.so" if os.environ.get("BDFB_LIBRARY") == "phases" else "libbdfb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run python -m paper_2011_12984_b300.build")

lib = C.CDLL(LIB_PATH)

SUCCESS = 0
TOO_MUCH_WORK = -1
ERR_FAILURE = -3
CONV_FAILURE = -4
LSETUP_FAIL = -6
LSOLVE_FAIL = -7
RHSFUNC_FAIL = -8
MEM_FAIL = -20
CUDA_FAIL = -21
ILL_INPUT = -22

MEM_HOST = 0
MEM_DEVICE = 1
ROBERTSON = 0
MASSACTION = 1
BRUSSELATOR3D = 2
BRUSSELATOR1D = 3
MASSACTION_SHARED = 4

_vp = C.c_void_p
_i64 = C.c_int64
_d = C.c_double
_i32 = C.c_int32


class Problem(C.Structure):
    _fields_ = [("kind", _i32), ("mem", _i32), ("ncell", _i64), ("n", _vp), ("y_off", _vp),
                ("rxn_off", _vp), ("reactants", _vp), ("products", _vp), ("k", _vp)]


class Stats(C.Structure):
    _fields_ = [("ncell", _i64), ("nsteps", _i64), ("nfevals", _i64), ("nlinsetups", _i64),
                ("nniters", _i64), ("nncfails", _i64), ("netfails", _i64), ("max_steps", _i64),
                ("min_steps", _i64), ("ncells_failed", _i64), ("nrefine", _i64),
                ("nrefine_fallback", _i64), ("last_kernel_ms", _d), ("nguess", _i64),
                ("nguess_fallback", _i64), ("graph_captures", _i64), ("graph_launches", _i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("bdfb_strerror", C.c_char_p, [C.c_int])
_sig("bdfb_version", C.c_int, [])
_sig("bdfb_nv_linear_sum", C.c_int, [_i64, _d, _vp, _d, _vp, _vp, _vp])
_sig("bdfb_nv_scale", C.c_int, [_i64, _d, _vp, _vp, _vp])
_sig("bdfb_nv_const", C.c_int, [_i64, _d, _vp, _vp])
_sig("bdfb_nv_abs", C.c_int, [_i64, _vp, _vp, _vp])
_sig("bdfb_nv_inv", C.c_int, [_i64, _vp, _vp, _vp])
_sig("bdfb_nv_add_const", C.c_int, [_i64, _vp, _d, _vp, _vp])
_sig("bdfb_nv_error_weights", C.c_int, [_i64, _d, _d, _vp, _vp, _vp])
_sig("bdfb_nv_linear_combination", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp])
_sig("bdfb_nv_scale_add_multi", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("bdfb_nv_dot_prod_multi", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("bdfb_nv_wrms_norm", C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp])
_sig("bdfb_nv_work_doubles", _i64, [_i64, C.c_int])
_sig("bdfb_batched_lu_factor", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp])
_sig("bdfb_batched_lu_solve", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp])
_sig("bdfb_batched_solve_mixed", C.c_int, [_i64, C.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("bdfb_sparse_create", C.c_int, [C.c_int, C.c_int, _vp, _vp, C.POINTER(_vp)])
_sig("bdfb_sparse_destroy", None, [_vp])
_sig("bdfb_sparse_lu_nnz", _i64, [_vp])
_sig("bdfb_sparse_load", C.c_int, [_vp, _i64, _vp, _vp, _vp])
_sig("bdfb_sparse_factor", C.c_int, [_vp, _i64, _vp, _vp, _vp])
_sig("bdfb_sparse_solve", C.c_int, [_vp, _i64, _vp, _vp, _vp])
_sig("bdfb_create", C.c_int, [C.POINTER(Problem), C.POINTER(_vp)])
_sig("bdfb_destroy", None, [_vp])
_sig("bdfb_set_stream", C.c_int, [_vp, _vp])
_sig("bdfb_set_tolerances", C.c_int, [_vp, _d, _d])
_sig("bdfb_set_option", C.c_int, [_vp, C.c_char_p, _i64])
_sig("bdfb_init", C.c_int, [_vp, _d, _vp, _i32])
_sig("bdfb_integrate", C.c_int, [_vp, _d, _vp, _vp, _i32])
_sig("bdfb_get_stats", C.c_int, [_vp, C.POINTER(Stats)])
_sig("bdfb_get_cell_stats", C.c_int, [_vp, _vp, _i32])
_sig("bdfb_get_op_profile", C.c_int, [_vp, _vp, _i32])
_sig("bdfb_get_mapping", C.c_int, [_vp, _vp, _vp])
_sig("bdfb_phase_cycles", C.c_int, [_vp, C.c_int, C.c_int])
_sig("bdfb_mlp_nparam", _i64, [])
_sig("bdfb_mlp_packed_bytes", _i64, [])
_sig("bdfb_mlp_pack", C.c_int, [_vp, _vp, _vp])
_sig("bdfb_mlp_forward", C.c_int, [_i64, _vp, _vp, _vp, _vp])
_sig("bdfb_mlp_loss_grad", C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp])
_sig("bdfb_mlp_train", C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, _i64,
                                 C.c_float, _vp])
_sig("bdfb_mlp_adam", C.c_int, [_vp, _vp, _vp, _vp, _i64, C.c_float, _vp])
_sig("bdfb_load_mlp", C.c_int, [_vp, _vp, _i64])
_sig("bdfb_set_record", C.c_int, [_vp, _vp, _vp, _i64, _vp])


# kinds of bdfb_get_op_profile, in order
OP_KINDS = ("wrms_norm", "dot_prod_multi", "linear_combination", "linear_sum", "predict", "accept",
            "rescale", "error_weights", "newton_update", "unscale", "rhs", "gmres_operator",
            "block_setup", "precondition_rhs")


class BdfbError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {lib.bdfb_strerror(code).decode()} ({code})")


def check(code, what=""):
    if code != SUCCESS:
        raise BdfbError(code, what)
    return code


PHASES = ("control", "predict", "jacobian", "factor_pivot", "factor_update", "rhs_rates", "rhs_gather",
          "triangular_solve", "residual", "refine_norms", "newton", "accept", "failure", "tile")


def phase_cycles(reset=True):
    """Cycles per step phase from a library built with the phase timers
    (``BDFB_LIBRARY=phases``), as a dict in ``PHASES`` order."""
    out = np.zeros(len(PHASES), dtype=np.uint64)
    r = lib.bdfb_phase_cycles(out.ctypes.data, len(PHASES), int(reset))
    if r < 0:
        raise BdfbError(r, "bdfb_phase_cycles (library built without the phase timers?)")
    return dict(zip(PHASES, (int(v) for v in out)))


def strerror(code):
    return lib.bdfb_strerror(code).decode()


# ------------------------------------------------------------------ helpers
def _torch():
    import torch
    return torch


def _dptr(t):
    """device pointer of a contiguous CUDA tensor (None -> NULL)"""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr_array(ts):
    return (_vp * len(ts))(*[_dptr(t) for t in ts])


def _f64_array(v):
    return (_d * len(v))(*[float(x) for x in v])


# ------------------------------------------------------------ vector ops
def nv_linear_sum(a, x, b, y, z, stream=None):
    return check(lib.bdfb_nv_linear_sum(x.numel(), a, _dptr(x), b, _dptr(y), _dptr(z), _stream(stream)),
                 "nv_linear_sum")


def nv_scale(c, x, z, stream=None):
    return check(lib.bdfb_nv_scale(z.numel(), c, _dptr(x), _dptr(z), _stream(stream)), "nv_scale")


def nv_const(c, z, stream=None):
    return check(lib.bdfb_nv_const(z.numel(), c, _dptr(z), _stream(stream)), "nv_const")


def nv_abs(x, z, stream=None):
    return check(lib.bdfb_nv_abs(z.numel(), _dptr(x), _dptr(z), _stream(stream)), "nv_abs")


def nv_inv(x, z, stream=None):
    return check(lib.bdfb_nv_inv(z.numel(), _dptr(x), _dptr(z), _stream(stream)), "nv_inv")


def nv_add_const(x, b, z, stream=None):
    return check(lib.bdfb_nv_add_const(z.numel(), _dptr(x), b, _dptr(z), _stream(stream)), "nv_add_const")


def nv_error_weights(rtol, atol, y, w, stream=None):
    return check(lib.bdfb_nv_error_weights(w.numel(), rtol, atol, _dptr(y), _dptr(w), _stream(stream)),
                 "nv_error_weights")


def nv_linear_combination(c, xs, z, stream=None):
    return check(lib.bdfb_nv_linear_combination(z.numel(), len(xs), _f64_array(c), _ptr_array(xs),
                                                _dptr(z), _stream(stream)), "nv_linear_combination")


def nv_scale_add_multi(a, x, ys, zs, stream=None):
    return check(lib.bdfb_nv_scale_add_multi(x.numel(), len(ys), _f64_array(a), _dptr(x),
                                             _ptr_array(ys), _ptr_array(zs), _stream(stream)),
                 "nv_scale_add_multi")


def nv_work(n, nv, device="cuda"):
    torch = _torch()
    return torch.zeros(int(lib.bdfb_nv_work_doubles(n, nv)), dtype=torch.float64, device=device)


def nv_dot_prod_multi(x, ys, out, work, stream=None):
    return check(lib.bdfb_nv_dot_prod_multi(x.numel(), len(ys), _dptr(x), _ptr_array(ys), _dptr(out),
                                            _dptr(work), _stream(stream)), "nv_dot_prod_multi")


def nv_wrms_norm(x, w, out, work, stream=None):
    return check(lib.bdfb_nv_wrms_norm(x.numel(), _dptr(x), _dptr(w), _dptr(out), _dptr(work),
                                       _stream(stream)), "nv_wrms_norm")


def batched_lu_factor(a, piv, info, stream=None):
    nb, n, _ = a.shape
    return check(lib.bdfb_batched_lu_factor(nb, n, _dptr(a), _dptr(piv), _dptr(info), _stream(stream)),
                 "batched_lu_factor")


def batched_lu_solve(lu, piv, b, stream=None):
    nb, n, _ = lu.shape
    return check(lib.bdfb_batched_lu_solve(nb, n, _dptr(lu), _dptr(piv), _dptr(b), _stream(stream)),
                 "batched_lu_solve")


def batched_solve_mixed(a, b, x, sweeps, stream=None):
    """FP32 LU + FP64 refinement of every block of a (nb, n, n) for rhs b (nb, n)"""
    nb, n, _ = a.shape
    return check(lib.bdfb_batched_solve_mixed(nb, n, _dptr(a), _dptr(b), _dptr(x), _dptr(sweeps),
                                              _stream(stream)), "batched_solve_mixed")


# ---------------------------------------------------- learned Newton guess
MLP_NI, MLP_NO = 12, 10
MLP_NPARAM = lib.bdfb_mlp_nparam()
MLP_PACKED_BYTES = lib.bdfb_mlp_packed_bytes()


def mlp_packed(device="cuda"):
    """uninitialised packed-network buffer (uint8 CUDA tensor, 16-byte aligned)"""
    return _torch().empty(MLP_PACKED_BYTES, dtype=_torch().uint8, device=device)


def mlp_pack(params, packed, stream=None):
    """FP32 parameters (CUDA, 5642) -> packed BF16 operand form"""
    return check(lib.bdfb_mlp_pack(_dptr(params), _dptr(packed), _stream(stream)), "mlp_pack")


def mlp_forward(X, packed, Y, stream=None):
    """Y (rows, 10) = net(X (rows, 12)), FP32 CUDA tensors"""
    return check(lib.bdfb_mlp_forward(X.shape[0], _dptr(X), _dptr(packed), _dptr(Y), _stream(stream)),
                 "mlp_forward")


def mlp_loss_grad(X, T, packed, grad, loss, stream=None):
    """grad (5642) += d loss / d params, loss (1) += mean squared error"""
    return check(lib.bdfb_mlp_loss_grad(X.shape[0], _dptr(X), _dptr(T), _dptr(packed), _dptr(grad),
                                        _dptr(loss), _stream(stream)), "mlp_loss_grad")


def mlp_adam(params, grad, m, v, t, lr=1e-3, stream=None):
    """one Adam step (step number t >= 1); grad is zeroed"""
    return check(lib.bdfb_mlp_adam(_dptr(params), _dptr(grad), _dptr(m), _dptr(v), int(t), float(lr),
                                   _stream(stream)), "mlp_adam")


def mlp_train(X, T, params, m, v, packed, grad, loss_hist, batch, nsteps, t0=0, lr=1e-3, stream=None):
    """nsteps Adam steps on minibatches of X, T (see bdfb_mlp_train)"""
    return check(lib.bdfb_mlp_train(X.shape[0], _dptr(X), _dptr(T), _dptr(params), _dptr(m), _dptr(v),
                                    _dptr(packed), _dptr(grad), _dptr(loss_hist), int(batch), int(nsteps),
                                    int(t0), float(lr), _stream(stream)), "mlp_train")


# ------------------------------------------------------------- integrator
class SparsePattern:
    """One sparsity pattern shared by every block of a block-diagonal matrix
    (``bdfb_sparse``).  rowptr / colind: host int32 CSR of the n x n block."""

    def __init__(self, n, rowptr, colind):
        self._rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        self._ci = np.ascontiguousarray(colind, dtype=np.int32)
        self.n = int(n)
        self.nnz = int(self._ci.size)
        h = _vp()
        check(lib.bdfb_sparse_create(self.n, self.nnz, self._rp.ctypes.data,
                                     self._ci.ctypes.data if self.nnz else None, C.byref(h)),
              "bdfb_sparse_create")
        self.h = h
        self.lu_nnz = int(lib.bdfb_sparse_lu_nnz(h))

    def load(self, a, lu, stream=None):
        """lu [lu_nnz, nb] <- a [nb, nnz] (CUDA float64 tensors)"""
        check(lib.bdfb_sparse_load(self.h, a.shape[0], _dptr(a), _dptr(lu), _stream(stream)), "bdfb_sparse_load")

    def factor(self, lu, info=None, stream=None):
        check(lib.bdfb_sparse_factor(self.h, lu.shape[1], _dptr(lu), _dptr(info), _stream(stream)),
              "bdfb_sparse_factor")

    def solve(self, lu, x, stream=None):
        """x [n, nb] <- M_b^{-1} x"""
        check(lib.bdfb_sparse_solve(self.h, lu.shape[1], _dptr(lu), _dptr(x), _stream(stream)),
              "bdfb_sparse_solve")

    def close(self):
        if self.h:
            lib.bdfb_sparse_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def species_major(problem, y=None):
    """cell-major values (the generators' layout) -> species-major (the
    layout of a shared-network integrator, y[s ncell + c])"""
    y = problem.y0 if y is None else y
    n = int(problem.n[0])
    return np.ascontiguousarray(np.asarray(y).reshape(problem.ncell, n).T).reshape(-1)


def cell_major(problem, y):
    n = int(problem.n[0])
    return np.ascontiguousarray(np.asarray(y).reshape(n, problem.ncell).T).reshape(-1)


class Integrator:
    """Owns a ``bdfb_ctx``.  ``problem`` is a generator problem (host arrays).
    ``shared_network=True`` (a problem whose cells all carry cell 0's network)
    creates a BDFB_MASSACTION_SHARED context: one copy of the network, states
    species-major (see ``species_major``), grouped integration on the shared
    sparse pattern, or with option grouped=0 every cell with its own step
    size and order on that pattern."""

    def __init__(self, problem, rtol=1e-6, atol=1e-10, stream=None, shared_network=False, **options):
        self._keep = []
        p = Problem()
        p.mem = MEM_HOST
        p.ncell = problem.npts if problem.kind in ("brusselator3d", "brusselator1d") else problem.ncell

        def host(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data

        if shared_network:
            if problem.kind != "massaction" or not getattr(problem, "shared", False):
                raise ValueError("shared_network needs a problem whose cells share one network")
            R = int(problem.rxn_off[1] - problem.rxn_off[0])
            p.kind = MASSACTION_SHARED
            p.n = host(problem.n[:1], np.int32)
            p.rxn_off = host([0, R], np.int64)
            p.reactants = host(problem.reactants[:R], np.uint8)
            p.products = host(problem.products[:R], np.uint8)
            p.k = host(problem.k[:R], np.float64)
        elif problem.kind == "robertson":
            p.kind = ROBERTSON
            p.k = host(problem.k, np.float64)
        elif problem.kind == "brusselator3d":
            p.kind = BRUSSELATOR3D
            p.ncell = problem.npts
            p.k = host([problem.A, problem.B, problem.eps, problem.D, float(problem.nx)], np.float64)
        elif problem.kind == "brusselator1d":
            p.kind = BRUSSELATOR1D
            p.k = host([problem.A, problem.B, problem.eps, problem.c, problem.length, float(problem.nx)],
                       np.float64)
        else:
            p.kind = MASSACTION
            p.n = host(problem.n, np.int32)
            p.y_off = host(problem.y_off, np.int64)
            p.rxn_off = host(problem.rxn_off, np.int64)
            p.reactants = host(problem.reactants, np.uint8)
            p.products = host(problem.products, np.uint8)
            p.k = host(problem.k, np.float64)
        h = _vp()
        check(lib.bdfb_create(C.byref(p), C.byref(h)), "bdfb_create")
        self._keep = []
        self.h = h
        if problem.kind in ("brusselator3d", "brusselator1d"):
            self.ncell, self.ny = 1, 3 * problem.npts    # one coupled system
        else:
            self.ncell = problem.ncell
            self.ny = int(problem.y_off[-1])
        self.shared = shared_network
        self.stat_rows = 1 if shared_network else self.ncell
        self.set_stream(stream)
        check(lib.bdfb_set_tolerances(self.h, rtol, atol), "bdfb_set_tolerances")
        for k, v in options.items():
            self.set_option(k, v)

    def set_stream(self, stream=None):
        self.stream = _stream(stream)
        check(lib.bdfb_set_stream(self.h, self.stream), "bdfb_set_stream")

    def set_option(self, key, value):
        check(lib.bdfb_set_option(self.h, key.encode(), int(value)), f"bdfb_set_option({key})")
        if self.shared and key == "grouped":          # per-cell mode: one row of counters per cell
            self.stat_rows = 1 if int(value) else self.ncell

    def set_tolerances(self, rtol, atol):
        check(lib.bdfb_set_tolerances(self.h, rtol, atol), "bdfb_set_tolerances")

    def init(self, t0, y0):
        """y0: CUDA tensor (device) or numpy array (host)."""
        if isinstance(y0, np.ndarray):
            y0 = np.ascontiguousarray(y0, dtype=np.float64)
            return check(lib.bdfb_init(self.h, t0, y0.ctypes.data, MEM_HOST), "bdfb_init")
        return check(lib.bdfb_init(self.h, t0, _dptr(y0), MEM_DEVICE), "bdfb_init")

    def integrate(self, tout, y, status=None):
        """y, status: CUDA tensors, or numpy arrays (host).  Returns the worst
        cell status (0 = all cells reached tout)."""
        if isinstance(y, np.ndarray):
            assert y.dtype == np.float64 and y.flags.c_contiguous
            sp = None
            if status is not None:
                assert status.dtype == np.int32 and status.flags.c_contiguous
                sp = status.ctypes.data
            r = lib.bdfb_integrate(self.h, tout, y.ctypes.data, sp, MEM_HOST)
        else:
            r = lib.bdfb_integrate(self.h, tout, _dptr(y), _dptr(status), MEM_DEVICE)
        if r < 0 and r in (MEM_FAIL, CUDA_FAIL, ILL_INPUT):
            raise BdfbError(r, "bdfb_integrate")
        return r

    def stats(self):
        s = Stats()
        check(lib.bdfb_get_stats(self.h, C.byref(s)), "bdfb_get_stats")
        return s.as_dict()

    def mapping(self):
        """(per size class (G, NMAX, cells) int32 [5, 3], autotune trial ms [5, 8])"""
        out = np.zeros((5, 3), np.int32)
        ms = np.zeros((5, 8), np.float32)
        check(lib.bdfb_get_mapping(self.h, out.ctypes.data, ms.ctypes.data), "bdfb_get_mapping")
        return out, ms

    def load_mlp(self, packed):
        """use a packed network (CUDA uint8 tensor; None detaches) for option predictor=1"""
        self._mlp = packed
        ptr = None if packed is None else _dptr(packed)
        n = 0 if packed is None else packed.numel() * packed.element_size()
        check(lib.bdfb_load_mlp(self.h, ptr, n), "bdfb_load_mlp")

    def set_record(self, x=None, t=None, count=None):
        """record accepted steps' (features, correction) pairs into x (cap, 12)
        and t (cap, 10) FP32 CUDA tensors; count: int64 CUDA tensor (1); x=None stops"""
        self._rec = (x, t, count)
        if x is None:
            return check(lib.bdfb_set_record(self.h, None, None, 0, None), "bdfb_set_record")
        return check(lib.bdfb_set_record(self.h, _dptr(x), _dptr(t), x.shape[0], _dptr(count)),
                     "bdfb_set_record")

    def op_profile(self):
        """grid contexts with option profile=1: {kind: (launches, ms, GB)}"""
        out = np.zeros(3 * len(OP_KINDS))
        n = lib.bdfb_get_op_profile(self.h, out.ctypes.data, len(OP_KINDS))
        check(n if n < 0 else 0, "bdfb_get_op_profile")
        return {k: (int(out[3 * i]), float(out[3 * i + 1]), float(out[3 * i + 2])) for i, k in enumerate(OP_KINDS)}

    def cell_stats(self):
        out = np.zeros((self.stat_rows, 8), np.int64)
        check(lib.bdfb_get_cell_stats(self.h, out.ctypes.data, MEM_HOST), "bdfb_get_cell_stats")
        return out

    def close(self):
        if getattr(self, "h", None):
            lib.bdfb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
