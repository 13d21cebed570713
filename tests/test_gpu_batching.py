"""GPU tests of the batching layer: the autotuner and CUDA graph replay.

* autotuned mappings meet the accuracy bar against the oracle and every size
  class gets a variant that can hold its cells;
* graph replay over several output times reproduces the launch-by-launch
  run bit for bit, patching tout without recapturing;
* cells of at most 16 species under the one-warp mapping run on the NMAX 16
  one-warp kernel and agree with the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2011_12984_b300 import bdfb, gen
from test_gpu_cells import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu
RTOL, ATOL, TEND = 1e-6, 1e-10, 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_mapping_accuracy(precision):
    p = gen.mass_action(100000, seed=31).subset(np.arange(2048))
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, autotune=1, precision=precision) as I:
        I.init(0.0, p.y0.copy())
        y = np.empty(p.y0.size)
        st = np.empty(p.ncell, np.int32)
        assert I.integrate(TEND, y, st) == 0 and np.all(st == 0)
        cs = I.cell_stats()
        mp, ms = I.mapping()
    check_against_oracle(p, TEND, RTOL, ATOL, y, cs)
    nmax = [4, 8, 16, 32, 56]
    for c in range(5):
        G, NMAX, cnt = mp[c]
        if cnt == 0:
            continue
        assert NMAX >= nmax[c] or (NMAX == 16 and c <= 2)
        assert G in (1, 4, 8, 16, 32)
        # the class's own variant was timed, unless it is the only one that
        # holds the class (the 56-species tiling)
        assert ms[c, c] > 0 or c == 4
    assert mp[:, 2].sum() == p.ncell
    s0 = np.add.reduceat(p.y0, p.y_off[:-1])
    assert np.max(np.abs(np.add.reduceat(y, p.y_off[:-1]) - s0)) <= 5e-11


def test_graph_replay_matches_direct_launches():
    p = gen.mass_action(100000, seed=32).subset(np.arange(1024))
    outs = [2.5e-4, 5e-4, 7.5e-4, 1e-3]
    res = {}
    for graph in (0, 1):
        with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, graph=graph) as I:
            I.init(0.0, torch.from_numpy(p.y0).cuda())
            y = torch.empty(p.y0.size, dtype=torch.float64, device="cuda")
            ys = []
            for t in outs:
                assert I.integrate(t, y) == 0
                ys.append(y.cpu().numpy().copy())
            res[graph] = (ys, I.cell_stats(), I.stats())
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[0][1], res[1][1])
    st = res[1][2]
    assert st["graph_captures"] == 1 and st["graph_launches"] == len(outs)
    assert res[0][2]["graph_launches"] == 0


def test_graph_recaptures_on_option_change():
    p = gen.mass_action(100000, seed=33).subset(np.arange(256))
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, graph=1) as I:
        I.init(0.0, p.y0.copy())
        y = np.empty(p.y0.size)
        assert I.integrate(5e-4, y) == 0
        I.set_tolerances(1e-7, 1e-11)
        assert I.integrate(1e-3, y) == 0
        assert I.stats()["graph_captures"] == 2


@pytest.mark.parametrize("sizes", [(3,), (10,)])
def test_one_warp_small_cell_kernel(sizes):
    """Cells of at most 16 species under mapping 32 run on the NMAX 16
    one-warp kernel (variant 5)."""
    p = gen.mass_action(100000, sizes=sizes, seed=34).subset(np.arange(512))
    ret, y, st, cs, _ = run_gpu(p, 0.0, TEND, RTOL, ATOL, mapping=32)
    assert ret == 0 and np.all(st == 0)
    with bdfb.Integrator(p, rtol=RTOL, atol=ATOL, mapping=32) as I:
        mp, _ = I.mapping()
    assert all(tuple(r[:2]) == (32, 16) for r in mp if r[2])
    check_against_oracle(p, TEND, RTOL, ATOL, y, cs)
