"""Edge cases of the per-cell and grouped paths: every size-class boundary
(cells of 2, 4, 5, 8, 9, 16, 17, 32, 33, 55 and 56 species, the largest and
smallest cell each tiling takes), an empty problem, and a ragged cell count,
against the oracle with the bars of the batched tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen
from test_gpu_cells import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu
SIZES = (2, 4, 5, 8, 9, 16, 17, 32, 33, 55, 56)


def boundary_problem(per_size=13):
    return gen.mass_action(per_size * len(SIZES), sizes=SIZES, seed=4242)


@pytest.mark.parametrize("mapping", [0, 32])
def test_every_size_class_boundary(mapping):
    p = boundary_problem()
    assert set(np.unique(p.n)) == set(SIZES)
    ret, y, st, cs, stats = run_gpu(p, 0.0, 1e-3, 1e-6, 1e-10, mapping=mapping)
    assert ret == 0 and np.all(st == 0)
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs)


def test_every_size_class_boundary_autotuned_mixed_precision():
    p = boundary_problem()
    ret, y, st, cs, stats = run_gpu(p, 0.0, 1e-3, 1e-6, 1e-10, precision=1, autotune=1)
    assert ret == 0 and np.all(st == 0)
    check_against_oracle(p, 1e-3, 1e-6, 1e-10, y, cs)


def test_empty_problem():
    p = gen.mass_action(8).subset(np.zeros(0, np.int64))
    with bdfb.Integrator(p) as I:
        I.init(0.0, np.zeros(0))
        assert I.integrate(1e-3, np.zeros(0), np.zeros(0, np.int32)) == 0
        assert I.stats()["nsteps"] == 0


def test_ragged_cell_count_grouped():
    """143 cells (no tile or block multiple), grouped mode, against the
    oracle's grouped integration"""
    p = boundary_problem(13)
    assert p.ncell == 143
    with bdfb.Integrator(p, rtol=1e-6, atol=1e-10, grouped=1) as I:
        I.init(0.0, torch.from_numpy(p.y0).cuda())
        y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
        assert I.integrate(1e-3, y) == 0
        stats = I.stats()
    y = y.cpu().numpy()
    yo, ro, so = oracle.integrate_cells_grouped(p, 0.0, 1e-3, 1e-6, 1e-10)
    assert ro == 0
    nst = stats["nsteps"] // p.ncell
    assert abs(nst / so[0] - 1.0) <= 0.05
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    s1 = np.add.reduceat(y, p.y_off[:-1])
    assert np.max(np.abs(s1 - s0) / np.abs(s0)) <= 1e-12
