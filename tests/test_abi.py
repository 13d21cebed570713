"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
symbol include/bdfb.h declares, and rejects bad arguments before touching the
GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bdfb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2011_12984_b300 import build
    path = build.build()
    return C.CDLL(path), path


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bdfb_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = declared()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(bdfb_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)


def test_strerror_and_version(lib):
    L, _ = lib
    L.bdfb_strerror.restype = C.c_char_p
    assert L.bdfb_strerror(0) == b"success"
    assert b"illegal" in L.bdfb_strerror(-22)
    assert L.bdfb_version() >= 100


def test_bad_arguments_rejected_without_gpu(lib):
    L, _ = lib
    ILL = -22
    L.bdfb_nv_linear_sum.argtypes = [C.c_int64, C.c_double, C.c_void_p, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    assert L.bdfb_nv_linear_sum(-1, 1.0, None, 1.0, None, None, None) == ILL
    assert L.bdfb_nv_linear_sum(0, 1.0, None, 1.0, None, None, None) == 0      # empty: no work
    L.bdfb_nv_linear_combination.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]
    assert L.bdfb_nv_linear_combination(10, 0, None, None, None, None) == ILL
    assert L.bdfb_nv_linear_combination(10, 17, None, None, None, None) == ILL
    L.bdfb_batched_lu_factor.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert L.bdfb_batched_lu_factor(4, 65, None, None, None, None) == ILL
    assert L.bdfb_batched_lu_factor(0, 10, None, None, None, None) == 0
    L.bdfb_create.argtypes = [C.c_void_p, C.c_void_p]
    assert L.bdfb_create(None, None) == ILL
    L.bdfb_set_option.argtypes = [C.c_void_p, C.c_char_p, C.c_int64]
    assert L.bdfb_set_option(None, b"mxstep", 5) == ILL
    L.bdfb_mlp_nparam.restype = C.c_int64
    assert L.bdfb_mlp_nparam() == 5642
    L.bdfb_mlp_packed_bytes.restype = C.c_int64
    assert L.bdfb_mlp_packed_bytes() % 16 == 0
    L.bdfb_mlp_forward.argtypes = [C.c_int64] + [C.c_void_p] * 4
    assert L.bdfb_mlp_forward(-1, None, None, None, None) == ILL
    assert L.bdfb_mlp_forward(0, None, None, None, None) == 0
    L.bdfb_mlp_loss_grad.argtypes = [C.c_int64] + [C.c_void_p] * 6
    assert L.bdfb_mlp_loss_grad(0, None, None, None, None, None, None) == ILL
    L.bdfb_mlp_pack.argtypes = [C.c_void_p] * 3
    assert L.bdfb_mlp_pack(None, None, None) == ILL
    L.bdfb_load_mlp.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    assert L.bdfb_load_mlp(None, None, 0) == ILL
    L.bdfb_set_record.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    assert L.bdfb_set_record(None, None, None, 0, None) == ILL


def test_binding_imports_and_fails_loudly_without_library(tmp_path):
    # the binding refuses to load when the shared library is missing
    src = open(os.path.join(ROOT, "paper_2011_12984_b300", "bdfb.py")).read()
    assert "raise ImportError" in src
    from paper_2011_12984_b300 import bdfb
    assert bdfb.lib is not None


def test_sparse_pattern_rejected_without_gpu(lib):
    """malformed shared patterns fail in the host analysis, before any device call"""
    L, _ = lib
    ILL = -22
    L.bdfb_sparse_create.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    h = C.c_void_p()
    rp = (C.c_int32 * 3)(0, 1, 2)
    ok_ci = (C.c_int32 * 2)(0, 1)
    assert L.bdfb_sparse_create(0, 0, rp, ok_ci, C.byref(h)) == ILL          # n < 1
    assert L.bdfb_sparse_create(2049, 0, rp, ok_ci, C.byref(h)) == ILL       # n too large
    bad_ci = (C.c_int32 * 2)(0, 2)
    assert L.bdfb_sparse_create(2, 2, rp, bad_ci, C.byref(h)) == ILL         # column out of range
    dup_rp = (C.c_int32 * 3)(0, 2, 2)
    dup_ci = (C.c_int32 * 2)(1, 1)
    assert L.bdfb_sparse_create(2, 2, dup_rp, dup_ci, C.byref(h)) == ILL     # duplicate entry
    bad_rp = (C.c_int32 * 3)(0, 2, 1)
    assert L.bdfb_sparse_create(2, 1, bad_rp, ok_ci, C.byref(h)) == ILL      # decreasing rowptr
    L.bdfb_sparse_factor.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    assert L.bdfb_sparse_factor(None, 4, None, None, None) == ILL


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mem", C.c_int32), ("ncell", C.c_int64), ("n", C.c_void_p),
                ("y_off", C.c_void_p), ("rxn_off", C.c_void_p), ("reactants", C.c_void_p),
                ("products", C.c_void_p), ("k", C.c_void_p)]


def test_shared_network_rejected_without_gpu(lib):
    """BDFB_MASSACTION_SHARED: a malformed network fails in the host checks"""
    L, _ = lib
    ILL = -22
    L.bdfb_create.argtypes = [C.POINTER(_Problem), C.POINTER(C.c_void_p)]

    def make(n, rxn, reac, prod, ncell=4, mem=0):
        arrs = dict(n=(C.c_int32 * 1)(n), rxn=(C.c_int64 * 2)(0, rxn),
                    reac=(C.c_uint8 * len(reac))(*reac), prod=(C.c_uint8 * len(prod))(*prod),
                    k=(C.c_double * max(rxn, 1))(*([1.0] * max(rxn, 1))))
        p = _Problem(4, mem, ncell, C.cast(arrs["n"], C.c_void_p), None, C.cast(arrs["rxn"], C.c_void_p),
                     C.cast(arrs["reac"], C.c_void_p), C.cast(arrs["prod"], C.c_void_p),
                     C.cast(arrs["k"], C.c_void_p))
        return p, arrs

    h = C.c_void_p()
    ok_r, ok_p = [0, 1, 255, 255], [2, 255, 255, 255]
    for bad in (dict(n=0, rxn=1, reac=ok_r, prod=ok_p),                 # no species
                dict(n=256, rxn=1, reac=ok_r, prod=ok_p),               # more than 255
                dict(n=3, rxn=1, reac=[0, 3, 255, 255], prod=ok_p),     # species out of range
                dict(n=3, rxn=1, reac=[1, 1, 255, 255], prod=ok_p),     # repeated reactant
                dict(n=3, rxn=1, reac=ok_r, prod=ok_p, mem=1),          # device arrays
                dict(n=3, rxn=1, reac=ok_r, prod=ok_p, ncell=0)):       # no cells
        p, keep = make(**bad)
        assert L.bdfb_create(C.byref(p), C.byref(h)) == ILL, bad


def test_phase_timers_absent_from_the_plain_build(lib):
    """the product library compiles the step-phase timers away: reading them
    is refused (without touching the GPU), whatever the buffer"""
    L, _ = lib
    f = L.bdfb_phase_cycles
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_int]
    out = (C.c_uint64 * 16)()
    assert f(out, 16, 0) == -22
    assert f(None, 16, 1) == -22
