"""The seeded input generators: published SplitMix64 output, reproducibility,
independence from chunking, and the distributions the recipes state."""
import numpy as np

from paper_2011_12984_b300 import gen


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (Vigna's reference code)
    assert int(gen._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_mass_action_reproducible_and_chunk_independent():
    a = gen.mass_action(300, seed=11)
    b = gen.mass_action(300, seed=11, chunk=7)
    for f in ("n", "y_off", "rxn_off", "reactants", "products", "k", "y0"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = gen.mass_action(300, seed=12)
    assert not np.array_equal(a.k, c.k)


def test_mass_action_distributions():
    p = gen.mass_action(4000, seed=1)
    counts = np.array([(p.n == s).sum() for s in (3, 10, 32, 54)])
    assert counts.sum() == 4000 and np.all(np.abs(counts - 1000) < 150)
    assert np.all(p.rxn_off[1:] - p.rxn_off[:-1] == 2 * p.n)
    lk = np.log10(p.k)
    assert lk.min() >= -2 and lk.max() < 8 and abs(lk.mean() - 3.0) < 0.1
    for c in range(0, 4000, 97):
        n = p.n[c]
        y = p.y0[p.y_off[c]:p.y_off[c + 1]]
        assert abs(y.sum() - 1.0) < 1e-14 and np.all(y > 0)
        for r in range(p.rxn_off[c], p.rxn_off[c + 1]):
            ra = p.reactants[r][p.reactants[r] != 255]
            pa = p.products[r][p.products[r] != 255]
            assert len(ra) == len(pa) and 2 <= len(ra) <= min(4, n)
            assert len(set(ra.tolist())) == len(ra) and len(set(pa.tolist())) == len(pa)
            assert ra.max() < n and pa.max() < n


def test_subset_repacks():
    p = gen.mass_action(50, seed=2)
    s = p.subset([3, 7])
    assert s.ncell == 2
    assert np.array_equal(s.y0[:p.n[3]], p.y0[p.y_off[3]:p.y_off[4]])
    assert np.array_equal(s.k[s.rxn_off[1]:], p.k[p.rxn_off[7]:p.rxn_off[8]])


def test_robertson_factors():
    p = gen.robertson(5000)
    f = p.k / np.array(gen.ROBERTSON_K)
    assert f.min() >= 0.5 and f.max() <= 2.0
    assert abs(np.log(f).mean()) < 0.02


def test_brusselator_noise():
    b = gen.brusselator3d(16)
    ss = np.repeat(np.array(gen.brusselator_steady_state(b.A, b.B, b.eps)), b.npts)
    rel = b.y0 / ss - 1.0
    assert np.max(np.abs(rel)) <= 0.01 and abs(rel.mean()) < 1e-3


def test_mass_action_shared_network():
    p = gen.mass_action_shared(50, n=10, seed=11)
    R = int(p.rxn_off[1])
    assert R == 20 and p.ncell == 50 and np.all(p.n == 10)
    for c in range(1, 50):        # one network for every cell
        sl = slice(p.rxn_off[c], p.rxn_off[c + 1])
        assert np.array_equal(p.reactants[sl], p.reactants[:R])
        assert np.array_equal(p.products[sl], p.products[:R])
        assert np.array_equal(p.k[sl], p.k[:R])
    # the initial states are those of unshared cells of the same size and seed
    q = gen.mass_action(50, sizes=(10,), seed=11)
    assert np.array_equal(p.y0, q.y0)
    assert np.allclose(np.add.reduceat(p.y0, p.y_off[:-1]), 1.0, rtol=0, atol=1e-14)


def test_banded_network_is_shared_banded_and_conservative():
    p = gen.mass_action_banded(5, n=64, window=6)
    q = gen.mass_action_banded(5, n=64, window=6)
    np.testing.assert_array_equal(p.reactants, q.reactants)       # deterministic
    np.testing.assert_array_equal(p.y0, q.y0)
    R = int(p.rxn_off[1])
    assert R == 128 and p.shared and p.subset([2, 3]).shared
    for c in range(1, 5):                                          # one network for all cells
        np.testing.assert_array_equal(p.reactants[c * R:(c + 1) * R], p.reactants[:R])
        np.testing.assert_array_equal(p.k[c * R:(c + 1) * R], p.k[:R])
    for ra, pa in zip(p.reactants[:R], p.products[:R]):
        r = [int(x) for x in ra if x != 255]
        s = [int(x) for x in pa if x != 255]
        assert len(r) == len(s) and len(set(r)) == len(r) and len(set(s)) == len(s)  # sum y conserved
        assert max(r + s) - min(r + s) < 6                         # within one window
    np.testing.assert_allclose(np.add.reduceat(p.y0, p.y_off[:-1]), 1.0, rtol=1e-14)
    assert not np.array_equal(p.y0[:64], p.y0[64:128])             # states differ per cell
