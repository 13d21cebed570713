"""GPU parity of the batched block LU (blocks of M = I - gamma J, Fig. 1 /
Sec. 5) against the oracle: same pivot rows, factors within rounding, same
zero-pivot report, and solves with normwise backward error <= 1e-12."""
import numpy as np
import pytest
import torch

import oracle

from paper_2011_12984_b300 import bdfb

pytestmark = pytest.mark.gpu


def blocks(nb, n, seed):
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((nb, n, n)) * 10.0 ** rng.uniform(-2, 5, size=(nb, n, n))
    return np.eye(n)[None] - 1e-3 * J


@pytest.mark.parametrize("n", [1, 2, 3, 10, 32, 54, 64])
@pytest.mark.parametrize("nb", [1, 37, 600])
def test_factor_and_solve(n, nb):
    M = blocks(nb, n, seed=n * 1000 + nb)
    a = torch.from_numpy(M).cuda()
    piv = torch.zeros((nb, n), dtype=torch.int32, device="cuda")
    info = torch.full((nb,), -5, dtype=torch.int32, device="cuda")
    bdfb.batched_lu_factor(a, piv, info)
    lu, pv, inf = a.cpu().numpy(), piv.cpu().numpy(), info.cpu().numpy()
    assert np.all(inf == 0)
    for b in range(0, nb, max(1, nb // 25)):
        olu, opiv, oinfo = oracle.lu_factor(M[b])
        assert oinfo == 0
        assert np.array_equal(pv[b], opiv)
        scale = np.max(np.abs(M[b]))
        assert np.max(np.abs(lu[b] - olu)) <= 1e-12 * max(1.0, scale) * n
    rhs = np.random.default_rng(n).standard_normal((nb, n))
    x = torch.from_numpy(rhs.copy()).cuda()
    bdfb.batched_lu_solve(a, piv, x)
    xs = x.cpu().numpy()
    for b in range(nb):
        r = M[b] @ xs[b] - rhs[b]
        eta = np.max(np.abs(r)) / (np.max(np.sum(np.abs(M[b]), axis=1)) * np.max(np.abs(xs[b]))
                                   + np.max(np.abs(rhs[b])))
        assert eta <= 1e-12, (b, eta)


def test_singular_block_reported():
    M = blocks(3, 3, 7)
    M[1] = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]])
    a = torch.from_numpy(M).cuda()
    piv = torch.zeros((3, 3), dtype=torch.int32, device="cuda")
    info = torch.zeros(3, dtype=torch.int32, device="cuda")
    bdfb.batched_lu_factor(a, piv, info)
    assert info.cpu().tolist() == [0, oracle.lu_factor(M[1])[2], 0]


def test_pivot_tie_goes_to_lowest_row():
    M = np.array([[[1.0, 2.0], [-1.0, 3.0]], [[0.0, 1.0], [2.0, 0.0]]])
    a = torch.from_numpy(M).cuda()
    piv = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    bdfb.batched_lu_factor(a, piv, info)
    assert piv.cpu().numpy()[:, 0].tolist() == [0, 1]
