"""GPU checks of the shared-pattern block-sparse matrices (bdfb_sparse: one
pattern for every block, Sec. 5) and of the grouped integrator of cells that
share one sparse network (BDFB_MASSACTION_SHARED).

Matrices: every block's solve has normwise backward error <= 1e-12 and
matches the oracle's pivoted dense LU solve to the conditioning; patterns
with fill (random, banded, arrow, dense, diagonal, 1 x 1), a ragged block
count, and a zero pivot that info reports.  Integrator: the oracle's grouped
integration (task-local Newton, dense LU per cell) on the same cells, with
the bar of the grouped-mode tests (oracle runs at rtol (1 +- 1e-12) set the
spread a global norm allows); Sigma y per cell to rounding; a full-size
run of 100 000 cells of 128 species checked on sampled cells.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu
THREADS = max(1, min(32, oracle.host_threads()))


def csr(mask):
    n = mask.shape[0]
    rowptr = np.zeros(n + 1, np.int32)
    cols = []
    for i in range(n):
        c = np.nonzero(mask[i])[0]
        cols.extend(c.tolist())
        rowptr[i + 1] = len(cols)
    return rowptr, np.asarray(cols, np.int32)


def patterns():
    rng = np.random.default_rng(3)
    out = {}
    m = rng.random((40, 40)) < 0.08
    np.fill_diagonal(m, True)
    out["random40"] = m
    n = 128
    i, j = np.indices((n, n))
    out["band128"] = np.abs(i - j) < 6
    a = np.eye(24, dtype=bool)
    a[0, :] = a[:, 0] = True            # arrow: fills completely
    out["arrow24"] = a
    out["dense16"] = np.ones((16, 16), bool)
    out["diag7"] = np.eye(7, dtype=bool)
    out["one"] = np.ones((1, 1), bool)
    return out


@pytest.mark.parametrize("name", list(patterns().keys()))
def test_factor_solve_backward_error(name):
    mask = patterns()[name]
    n = mask.shape[0]
    rowptr, colind = csr(mask)
    nb = 1001                                   # ragged against the 128-thread blocks
    rng = np.random.default_rng(7)
    vals = rng.uniform(-1, 1, (nb, colind.size))
    diag_e = [rowptr[i] + np.nonzero(colind[rowptr[i]:rowptr[i + 1]] == i)[0][0] for i in range(n)]
    vals[:, diag_e] += n * 0.6 * np.sign(vals[:, diag_e]) + 0.5   # pivots away from zero
    sp = bdfb.SparsePattern(n, rowptr, colind)
    assert sp.lu_nnz >= colind.size
    a = torch.from_numpy(vals).cuda()
    lu = torch.empty((sp.lu_nnz, nb), dtype=torch.float64, device="cuda")
    info = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
    sp.load(a, lu)
    sp.factor(lu, info)
    b = rng.uniform(-1, 1, (nb, n))
    x = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    sp.solve(lu, x)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    X = x.cpu().numpy().T
    worst = 0.0
    for blk in range(0, nb, 97):
        A = np.zeros((n, n))
        for r in range(n):
            A[r, colind[rowptr[r]:rowptr[r + 1]]] = vals[blk, rowptr[r]:rowptr[r + 1]]
        res = A @ X[blk] - b[blk]
        be = np.abs(res).max() / (np.abs(A).sum(axis=1).max() * np.abs(X[blk]).max() + np.abs(b[blk]).max())
        worst = max(worst, be)
        lu_o, piv, inf = oracle.lu_factor(A)
        assert inf == 0
        xo = oracle.lu_solve(lu_o, piv, b[blk])
        cond = np.linalg.cond(A)
        assert np.abs(X[blk] - xo).max() <= 1e-14 * cond * max(1.0, np.abs(xo).max())
    assert worst <= 1e-12, worst
    sp.close()


def test_zero_pivot_reported():
    mask = np.ones((2, 2), bool)
    rowptr, colind = csr(mask)
    sp = bdfb.SparsePattern(2, rowptr, colind)
    vals = np.array([[0.0, 1.0, 1.0, 0.0], [2.0, 1.0, 1.0, 2.0]])   # block 0 needs a row swap
    lu = torch.empty((sp.lu_nnz, 2), dtype=torch.float64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    sp.load(torch.from_numpy(vals).cuda(), lu)
    sp.factor(lu, info)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [1, 0]


def rms(e):
    return float(np.sqrt(np.mean(e * e)))


def run_shared(p, tout, rtol, atol):
    with bdfb.Integrator(p, rtol=rtol, atol=atol, shared_network=True) as I:
        I.init(0.0, torch.from_numpy(bdfb.species_major(p)).cuda())
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        st = torch.empty(p.ncell, dtype=torch.int32, device="cuda")
        r = I.integrate(tout, y, st)
        torch.cuda.synchronize()
        assert r == 0, bdfb.strerror(r)
        assert np.all(st.cpu().numpy() == 0)
        return bdfb.cell_major(p, y.cpu().numpy()), I.stats(), I.cell_stats()[0]


@pytest.mark.parametrize("which", ["banded128", "shared10", "shared40"])
def test_grouped_shared_network_against_oracle(which):
    """banded128 takes the register-window solves; shared10 and shared40 (a
    random network: general pattern with fill) the general schedule"""
    if which == "banded128":
        p = gen.mass_action_banded(96, n=128)
    elif which == "shared10":
        p = gen.mass_action_shared(1000, n=10)
    else:
        p = gen.mass_action_shared(200, n=40)
    tout, rtol, atol = 1e-3, 1e-6, 1e-10
    y, stats, row = run_shared(p, tout, rtol, atol)
    yt, stt, _ = oracle.integrate_cells(p, 0.0, tout, 1e-10, 1e-14, threads=THREADS)
    assert np.all(stt == 0)
    w = lambda v: np.abs(v - yt) / (rtol * np.abs(yt) + atol)
    worst_max = worst_rms = 0.0
    runs = []
    for f in (1.0, 1.0 + 1e-12, 1.0 - 1e-12):
        yo, ro, s = oracle.integrate_cells_grouped(p, 0.0, tout, rtol * f, atol)
        assert ro == 0
        runs.append(s)
        worst_max, worst_rms = max(worst_max, w(yo).max()), max(worst_rms, rms(w(yo)))
    runs = np.array(runs)
    eg = w(y)
    assert eg.max() <= max(10.0, 2.0 * worst_max), (eg.max(), worst_max)
    assert rms(eg) <= max(0.05, 1.5 * worst_rms), (rms(eg), worst_rms)
    # counts within 5% / 10% of the range the three oracle runs span
    nst = stats["nsteps"] // p.ncell
    assert 0.95 * runs[:, 0].min() <= nst <= 1.05 * runs[:, 0].max(), (nst, runs[:, 0])
    assert 0.9 * runs[:, 3].min() <= stats["nniters"] <= 1.1 * runs[:, 3].max(), (stats["nniters"], runs[:, 3])
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12
    if which == "banded128":
        assert row[6] >= row[7] > 0          # LU entries with fill >= entries of M


def test_full_size_100k_cells_128_species():
    p = gen.mass_action_banded(100_000, n=128)
    y, stats, row = run_shared(p, 1e-3, 1e-6, 1e-10)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12
    cells = np.sort(np.random.default_rng(5).choice(p.ncell, 64, replace=False))
    sub = p.subset(cells)
    yt, stt, _ = oracle.integrate_cells(sub, 0.0, 1e-3, 1e-10, 1e-14, threads=THREADS)
    assert np.all(stt == 0)
    ys = np.concatenate([y[p.y_off[c]:p.y_off[c + 1]] for c in cells])
    e = np.abs(ys - yt) / (1e-6 * np.abs(yt) + 1e-10)
    # one error norm over all species bounds their RMS, not the largest one:
    # grouped oracle runs of 512-768 mixed cells reach 11-52 weighted units
    assert rms(e) <= 1.0 and e.max() <= 50.0, (rms(e), e.max())
    assert stats["max_steps"] == stats["min_steps"] > 0


# ------------------------------------ per-cell step control on the shared pattern
def run_percell(p, tout, rtol, atol, interp=0, y0=None):
    """option grouped=0: every cell with its own step size and order, one
    thread per cell on the shared sparse LU; returns cell-major y, statuses,
    per-cell counters and totals"""
    with bdfb.Integrator(p, rtol=rtol, atol=atol, shared_network=True, grouped=0, interp=interp) as I:
        y0 = p.y0 if y0 is None else y0
        I.init(0.0, torch.from_numpy(bdfb.species_major(p, y0)).cuda())
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        st = torch.empty(p.ncell, dtype=torch.int32, device="cuda")
        r = I.integrate(tout, y, st)
        torch.cuda.synchronize()
        return r, bdfb.cell_major(p, y.cpu().numpy()), st.cpu().numpy(), I.cell_stats(), I.stats()


@pytest.mark.parametrize("which", ["shared10", "shared40"])
def test_percell_shared_network_against_oracle(which):
    """cell by cell against the oracle's per-cell integration of the same
    cells (dense pivoted LU there, the shared sparse LU here: the same method
    up to rounding) with the tiers of the per-cell parity tests"""
    from test_gpu_cells import check_against_oracle
    p = gen.mass_action_shared(1000, n=10) if which == "shared10" else gen.mass_action_shared(200, n=40)
    r, y, st, cs, stats = run_percell(p, 1e-3, 1e-6, 1e-10)
    assert r == 0 and np.all(st == 0)
    assert cs.shape == (p.ncell, 8) and stats["nsteps"] == cs[:, 0].sum()
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    assert np.max(np.abs(np.add.reduceat(y, p.y_off[:-1]) - s0)) <= 5e-11
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs, min_seq=0.4)


def test_percell_banded_128_against_oracle():
    """the 128-species banded network (the per-cell dense path holds at most
    56 species): per cell against the oracle"""
    from test_gpu_cells import check_against_oracle
    p = gen.mass_action_banded(96, n=128)
    r, y, st, cs, _ = run_percell(p, 1e-3, 1e-6, 1e-10)
    assert r == 0 and np.all(st == 0)
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs, min_seq=0.4)


def test_percell_interp_and_continuation():
    """interpolated output against the oracle in the same mode; a later call
    continues from where the cells stopped"""
    from test_gpu_cells import check_against_oracle
    p = gen.mass_action_shared(512, n=10, seed=31)
    r, y, st, cs, _ = run_percell(p, 1e-3, 1e-6, 1e-10, interp=1)
    assert r == 0 and np.all(st == 0)
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs, min_seq=0.4, interp=True)
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, shared_network=True, grouped=0) as I:
        I.init(0.0, bdfb.species_major(p))
        y1 = np.empty(p.y0.size)
        assert I.integrate(5e-4, y1) == 0 and I.integrate(1e-3, y1) == 0
    # two calls (a fresh Jacobian and a clamped step at 5e-4) make another
    # valid integration: each cell within the range of the oracle's errors
    yt, _, _ = oracle.integrate_cells(p, 0.0, 1e-3, 1e-10, 1e-14, threads=THREADS)
    yo, _, _ = oracle.integrate_cells(p, 0.0, 1e-3, 1e-6, 1e-10, threads=THREADS)
    w = lambda v: np.maximum.reduceat(np.abs(v - yt) / (1e-6 * np.abs(yt) + 1e-10), p.y_off[:-1])
    assert w(bdfb.cell_major(p, y1)).max() <= max(10.0, 1.5 * w(yo).max())


def test_percell_failing_cell_is_isolated():
    """a cell whose state is NaN fails its right-hand side alone"""
    p = gen.mass_action_shared(64, n=10, seed=32)
    y0 = p.y0.copy()
    y0[p.y_off[5]] = np.nan
    r, y, st, cs, _ = run_percell(p, 1e-3, 1e-6, 1e-10, y0=y0)
    assert r == bdfb.RHSFUNC_FAIL and st[5] == bdfb.RHSFUNC_FAIL
    assert np.all(np.delete(st, 5) == 0)


def test_percell_full_size_100k_cells_128_species():
    p = gen.mass_action_banded(100_000, n=128)
    r, y, st, cs, stats = run_percell(p, 1e-3, 1e-6, 1e-10)
    assert r == 0 and np.all(st == 0)
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    assert np.max(np.abs(np.add.reduceat(y, p.y_off[:-1]) - s0) / np.abs(s0)) <= 1e-12
    cells = np.sort(np.random.default_rng(6).choice(p.ncell, 64, replace=False))
    sub = p.subset(cells)
    ys = np.concatenate([y[p.y_off[c]:p.y_off[c + 1]] for c in cells])
    yt, stt, _ = oracle.integrate_cells(sub, 0.0, 1e-3, 1e-10, 1e-14, threads=THREADS)
    yo, so, _ = oracle.integrate_cells(sub, 0.0, 1e-3, 1e-6, 1e-10, threads=THREADS)
    assert np.all(stt == 0) and np.all(so == 0)
    w = lambda v: np.maximum.reduceat(np.abs(v - yt) / (1e-6 * np.abs(yt) + 1e-10), sub.y_off[:-1])
    eg, eo = w(ys), w(yo)
    assert np.all(eg <= np.maximum(3.0 * eo + 10.0, max(10.0, 1.5 * eo.max())))
    assert stats["max_steps"] >= stats["min_steps"] > 0
