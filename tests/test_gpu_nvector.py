"""GPU parity of the fused NVECTOR kernels against the oracle (Sec. 4 streaming
and reduction operations).  Bar: every output within 1e-14 of the sum of the
absolute values of the terms that form it (the kernels differ from the oracle
only by fused multiply-adds and summation order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu
DEV = "cuda"
SIZES = [0, 1, 2, 7, 1000, 4097, 262147]


def to_dev(a, offset=0):
    """device copy; offset=1 places it 8 bytes past a 16-byte boundary"""
    t = torch.empty(a.size + offset, dtype=torch.float64, device=DEV)
    t[offset:] = torch.from_numpy(np.ascontiguousarray(a))
    return t[offset:]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off", [0, 1])
def test_linear_sum(n, off):
    x, y = gen.uniform_vectors(n, 2, seed=n + 1)
    dx, dy = to_dev(x, off), to_dev(y, off)
    dz = to_dev(np.zeros(n), off)
    bdfb.nv_linear_sum(1.5, dx, -0.25, dy, dz)
    ref = oracle.linear_sum(1.5, x, -0.25, y)
    assert np.all(np.abs(dz.cpu().numpy() - ref) <= 1e-14 * (np.abs(1.5 * x) + np.abs(0.25 * y)))
    bdfb.nv_linear_sum(2.0, dx, 1.0, dy, dx)                 # z aliases x
    assert np.all(np.abs(dx.cpu().numpy() - (2 * x + y)) <= 1e-14 * (np.abs(2 * x) + np.abs(y)))


@pytest.mark.parametrize("a,b", [(0.75, 1.0), (0.75, -1.0), (1.0, -0.3), (-1.0, 0.3), (1.0, 1.0), (-1.0, -1.0)])
def test_linear_sum_unit_coefficients(a, b):
    """the one-operation forms for a coefficient of +-1 (sums, differences,
    axpy) against the oracle, with an odd length (vector body and tail)"""
    n = 262147
    x, y = gen.uniform_vectors(n, 2, seed=7)
    dz = to_dev(np.zeros(n))
    bdfb.nv_linear_sum(a, to_dev(x), b, to_dev(y), dz)
    ref = oracle.linear_sum(a, x, b, y)
    assert np.all(np.abs(dz.cpu().numpy() - ref) <= 1e-14 * (np.abs(a * x) + np.abs(b * y)))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("nv", [1, 3, 6, 16])
def test_linear_combination(n, nv):
    xs = gen.uniform_vectors(n, nv, seed=100 + n)
    c = np.linspace(-2.0, 3.0, nv)
    dz = to_dev(np.zeros(n), nv % 2)
    bdfb.nv_linear_combination(c, [to_dev(x, nv % 2) for x in xs], dz)
    ref = oracle.linear_combination(c, list(xs))
    scale = sum(np.abs(c[j] * xs[j]) for j in range(nv))
    assert np.all(np.abs(dz.cpu().numpy() - ref) <= 1e-14 * scale)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("nv", [1, 2, 6, 16])
def test_scale_add_multi(n, nv):
    v = gen.uniform_vectors(n, nv + 1, seed=200 + n)
    x, ys = v[0], list(v[1:])
    a = np.linspace(0.5, -1.5, nv)
    dys = [to_dev(y) for y in ys]
    dzs = [to_dev(np.zeros(n)) for _ in ys]
    bdfb.nv_scale_add_multi(a, to_dev(x), dys, dzs)
    refs = oracle.scale_add_multi(a, x, ys)
    for j in range(nv):
        assert np.all(np.abs(dzs[j].cpu().numpy() - refs[j]) <= 1e-14 * (np.abs(a[j] * x) + np.abs(ys[j])))
    bdfb.nv_scale_add_multi(a, to_dev(x), dys, dys)          # z_j aliases y_j
    for j in range(nv):
        assert np.all(np.abs(dys[j].cpu().numpy() - refs[j]) <= 1e-14 * (np.abs(a[j] * x) + np.abs(ys[j])))


@pytest.mark.parametrize("n", SIZES + [5_000_001])
@pytest.mark.parametrize("off", [0, 1])
def test_dot_prod_multi(n, off):
    nv = 5
    v = gen.uniform_vectors(n, nv + 1, seed=300 + n)
    x, ys = v[0], list(v[1:])
    out = torch.zeros(nv, dtype=torch.float64, device=DEV)
    work = bdfb.nv_work(n, nv)
    for rep in range(2):                       # the workspace is reusable
        bdfb.nv_dot_prod_multi(to_dev(x, off), [to_dev(y, off) for y in ys], out, work)
        d, sabs = oracle.dot_prod_multi(x, ys)
        assert np.all(np.abs(out.cpu().numpy() - d) <= 1e-14 * sabs + 1e-300)


@pytest.mark.parametrize("n", SIZES + [5_000_001])
def test_wrms_norm(n):
    x, y = gen.uniform_vectors(n, 2, seed=400 + n)
    w = 1.0 / (1e-6 * np.abs(y) + 1e-10)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    work = bdfb.nv_work(n, 1)
    bdfb.nv_wrms_norm(to_dev(x), to_dev(w), out, work)
    ref = oracle.wrms_norm(x, w) if n else 0.0
    assert abs(out.item() - ref) <= 1e-14 * ref + 1e-300


def test_large_vectors_sampled():
    """At the benchmark length (N = 2^25 + 1) elementwise results are checked
    on sampled indices against the per-element definition, reductions in full."""
    n = (1 << 25) + 1
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.rand(n, dtype=torch.float64, generator=g) * 2 - 1
    y = torch.rand(n, dtype=torch.float64, generator=g) * 2 - 1
    dx, dy = x.to(DEV), y.to(DEV)
    dz = torch.empty_like(dx)
    bdfb.nv_linear_combination([0.5, -1.0, 2.0], [dx, dy, dx], dz)
    idx = np.random.default_rng(1).integers(0, n, 20000)
    xs, ys = x.numpy()[idx], y.numpy()[idx]
    ref = oracle.linear_combination([0.5, -1.0, 2.0], [xs, ys, xs])
    assert np.all(np.abs(dz.cpu().numpy()[idx] - ref) <= 1e-14 * (2.5 * np.abs(xs) + np.abs(ys)))
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    bdfb.nv_dot_prod_multi(dx, [dy, dx], out, bdfb.nv_work(n, 2))
    d, s = oracle.dot_prod_multi(x.numpy(), [y.numpy(), x.numpy()])
    assert np.all(np.abs(out.cpu().numpy() - d) <= 1e-14 * s)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off", [0, 1])
def test_support_ops(n, off):
    """Scale, Const, Abs, Inv, AddConst: one correctly rounded operation per
    element, so bitwise equal to the oracle; error weights within 2 ulp (the
    kernel may fuse rtol |y| + atol into one multiply-add, and takes the
    reciprocal by Newton-Raphson from an FP32 seed, within half an ulp)."""
    (x,) = gen.uniform_vectors(n, 1, seed=n + 7)
    x = x + np.sign(x) * 1e-3                      # keep 1/x finite
    dx = to_dev(x, off)
    dz = to_dev(np.zeros(n), off)
    bdfb.nv_scale(-2.5, dx, dz)
    assert np.array_equal(dz.cpu().numpy(), oracle.scale(-2.5, x))
    bdfb.nv_const(3.25, dz)
    assert np.array_equal(dz.cpu().numpy(), oracle.const(3.25, n))
    bdfb.nv_abs(dx, dz)
    assert np.array_equal(dz.cpu().numpy(), oracle.abs_(x))
    bdfb.nv_inv(dx, dz)
    assert np.array_equal(dz.cpu().numpy(), oracle.inv(x))
    bdfb.nv_add_const(dx, 0.125, dz)
    assert np.array_equal(dz.cpu().numpy(), oracle.add_const(x, 0.125))
    bdfb.nv_error_weights(1e-6, 1e-10, dx, dz)
    w = oracle.error_weights(1e-6, 1e-10, x)
    assert np.all(np.abs(dz.cpu().numpy() - w) <= 4.5e-16 * w)
    bdfb.nv_scale(0.5, dx, dx)                     # z aliases x
    assert np.array_equal(dx.cpu().numpy(), oracle.scale(0.5, x))
