"""Mixed precision (FP32 factorisation, FP64 iterative refinement).

* The dense-block solve reaches normwise backward error <= 1e-12 in FP64 on
  blocks M = I - gamma J shaped like the integrator's, and agrees with the
  oracle's FP64 LU solve to the conditioning the backward error allows.
* The integrator with FP32 factors meets the same final-state bar as the FP64
  form on n = 54 mass-action cells, with the FP64 history, error test and
  convergence test unchanged.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

from test_gpu_cells import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu


def blocks(nb, n, seed, scale=1e-3):
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((nb, n, n)) * 10.0 ** rng.uniform(-2, 4, size=(nb, n, n))
    return np.eye(n)[None] - scale * J


def backward_error(M, x, b):
    """normwise backward error |M x - b|_inf / (|M|_inf |x|_inf + |b|_inf)"""
    r = M @ x - b
    return np.max(np.abs(r)) / (np.max(np.sum(np.abs(M), axis=1)) * np.max(np.abs(x))
                                + np.max(np.abs(b)))


@pytest.mark.parametrize("n", [1, 3, 10, 32, 54, 64])
def test_refined_solve_backward_error(n):
    """every block reaches backward error <= 1e-12, by refinement or, where
    refinement stalls, by the FP64 fallback (sweeps 0); the fallback stays rare"""
    nb = 300
    M = blocks(nb, n, seed=7 * n)
    rhs = np.random.default_rng(n).standard_normal((nb, n))
    x = torch.zeros((nb, n), dtype=torch.float64, device="cuda")
    sw = torch.zeros(nb, dtype=torch.int32, device="cuda")
    bdfb.batched_solve_mixed(torch.from_numpy(M).cuda(), torch.from_numpy(rhs).cuda(), x, sw)
    xs, sws = x.cpu().numpy(), sw.cpu().numpy()
    assert np.all(sws >= 0), np.unique(sws, return_counts=True)
    assert (sws == 0).mean() <= 0.05, np.unique(sws, return_counts=True)
    for b in range(nb):
        eta = backward_error(M[b], xs[b], rhs[b])
        assert eta <= 1e-12, (b, eta, sws[b])
        lu, piv, _ = oracle.lu_factor(M[b])
        xo = oracle.lu_solve(lu, piv, rhs[b])
        cond = np.linalg.cond(M[b], np.inf)
        assert np.max(np.abs(xs[b] - xo)) <= 1e-11 * cond * np.max(np.abs(xo)) + 1e-300


def test_ill_conditioned_blocks_fall_back_to_fp64():
    """FP32 factors cannot refine a block with condition ~1e12: the solve
    falls back to FP64 LU (sweeps 0) and still meets the 1e-12 backward error,
    beside a well-conditioned block refined in the same launch"""
    n = 8
    U, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, n)))
    V, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, n)))
    M = np.stack([U @ np.diag(np.logspace(0, -12, n)) @ V.T, np.eye(n) + 0.1 * U])
    rhs = np.ones((2, n))
    x = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    sw = torch.zeros(2, dtype=torch.int32, device="cuda")
    bdfb.batched_solve_mixed(torch.from_numpy(M).cuda(), torch.from_numpy(rhs).cuda(), x, sw)
    sws, xs = sw.cpu().numpy(), x.cpu().numpy()
    assert sws[0] == 0 and sws[1] >= 1
    for b in range(2):
        assert backward_error(M[b], xs[b], rhs[b]) <= 1e-12


def test_singular_block_reported():
    """an exactly singular block: both factorisations meet a zero pivot (-2)"""
    n = 4
    M = np.ones((1, n, n))
    x = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    sw = torch.zeros(1, dtype=torch.int32, device="cuda")
    bdfb.batched_solve_mixed(torch.from_numpy(M).cuda(), torch.ones((1, n), dtype=torch.float64).cuda(), x, sw)
    assert sw.item() == -2


def test_mixed_integrator_n54():
    p = gen.mass_action(2048, sizes=(54,), seed=21).subset(np.arange(384))
    ret, y, st, cs, stats = run_gpu(p, 0.0, 1e-3, 1e-6, 1e-10, precision=1)
    assert ret == 0 and np.all(st == 0)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0)) <= 5e-11
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs)
    assert stats["nrefine"] >= stats["nniters"]          # at least one sweep per solve
    assert stats["nrefine_fallback"] <= 0.05 * stats["nlinsetups"]


def test_mixed_one_warp_per_cell():
    """precision 1 with mapping 32 (every cell on a one-warp-per-cell kernel,
    including the 54-species class's range): the FP64 fallback workspace of the
    kernel actually launched exists, and the run meets the same bar"""
    p = gen.mass_action(100000, seed=22).subset(np.arange(768))
    ret, y, st, cs, stats = run_gpu(p, 0.0, 1e-3, 1e-6, 1e-10, precision=1, mapping=32)
    assert ret == 0 and np.all(st == 0)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    assert np.max(np.abs(np.add.reduceat(y, p.y_off[:-1]) - s0)) <= 5e-11
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs)
    # cells small enough for the 32-species kernel only (its workspace is
    # then the only one), with FP32 factors for the small cells too
    q = gen.mass_action(100000, sizes=(3, 10, 32), seed=23).subset(np.arange(512))
    ret, y, st, cs, stats = run_gpu(q, 0.0, 1e-3, 1e-6, 1e-10, precision=1, mapping=32, mixed_small=1)
    assert ret == 0 and np.all(st == 0)
    assert stats["nrefine"] >= stats["nniters"]
    check_against_oracle(q, 1e-3, 1e-6, 1e-10, y, cs)


@pytest.mark.parametrize("mapping", [0, 32])
def test_mixed_factors_only_the_largest_cells_by_default(mapping):
    """precision 1 factors in FP32 only the cells of more than 32 species
    (their kernels): a batch of smaller cells runs FP64 factors (no refinement
    sweep) unless mixed_small is set; both meet the same bar"""
    q = gen.mass_action(100000, sizes=(3, 10, 32), seed=24).subset(np.arange(384))
    for small in (0, 1):
        ret, y, st, cs, stats = run_gpu(q, 0.0, 1e-3, 1e-6, 1e-10, precision=1, mapping=mapping,
                                        mixed_small=small)
        assert ret == 0 and np.all(st == 0)
        if small:
            assert stats["nrefine"] >= stats["nniters"]
        else:
            assert stats["nrefine"] == 0 and stats["nrefine_fallback"] == 0
        check_against_oracle(q, 1e-3, 1e-6, 1e-10, y, cs)


def test_mixed_small_option_rejected_off_mass_action():
    with bdfb.Integrator(gen.robertson(4)) as I:
        with pytest.raises(bdfb.BdfbError):
            I.set_option("mixed_small", 1)
        I.set_option("mixed_small", 0)


def test_mixed_rejected_for_robertson():
    p = gen.robertson(4)
    with bdfb.Integrator(p) as I:
        with pytest.raises(bdfb.BdfbError):
            I.set_option("precision", 1)


def test_mixed_full_size_sampled():
    """The 262 144-cell, 54-species workload in both factorisations, as the
    benchmark runs it: every cell succeeds and conserves sum y; 128 sampled
    cells against the truth; the two precisions agree to the tolerance."""
    p = gen.mass_action(262144, sizes=(54,), seed=gen.DEFAULT_SEED + 7)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    cells = np.sort(np.random.default_rng(5).choice(p.ncell, 128, replace=False))
    ys = {}
    for prec in (0, 1):
        ret, y, st, cs, stats = run_gpu(p, 0.0, 1e-3, 1e-6, 1e-10, precision=prec)
        assert ret == 0 and np.all(st == 0)
        assert np.max(np.abs(np.add.reduceat(y, p.y_off[:-1]) - s0)) <= 5e-11
        ysub = np.concatenate([y[p.y_off[c]:p.y_off[c + 1]] for c in cells])
        check_against_oracle(p.subset(cells), 1e-3, 1e-6, 1e-10, ysub, cs[cells])
        ys[prec] = y
    w = 1e-6 * np.abs(ys[0]) + 1e-10
    assert np.median(np.abs(ys[1] - ys[0]) / w) <= 3.0
