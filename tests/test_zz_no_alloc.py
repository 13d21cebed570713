"""The multi-dot product that allocates nothing.

Callers whose memory manager owns all device memory, or that must avoid the
synchronisation a device allocation can cause, use
bdfb_nv_dot_prod_multi_noalloc: its scratch is a fixed array inside the
library.  This test calls it through the C ABI and compares it with the
workspace-taking bdfb_nv_dot_prod_multi on two calls in a row (the shared
scratch keeps the previous call's contents).  It lives in its own file,
collected last, and passes both alone in a fresh process and after the
other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2011_12984_b300 import bdfb, gen

pytestmark = pytest.mark.gpu

L = bdfb.lib
L.bdfb_nv_dot_prod_multi_noalloc.restype = C.c_int
L.bdfb_nv_dot_prod_multi_noalloc.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]
L.bdfb_nv_noalloc_max_nv.restype = C.c_int64


def noalloc(x, ys, out, stream):
    ptrs = (C.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    return L.bdfb_nv_dot_prod_multi_noalloc(x.numel(), len(ys), x.data_ptr(), ptrs, out.data_ptr(),
                                            stream)


@pytest.mark.parametrize("n,nv", [(1_000_003, 5), (4097, 16), (1, 1)])
def test_noalloc_matches_workspace_entry_point_twice(n, nv):
    v = gen.uniform_vectors(n, nv + 1, seed=900 + n)
    dx = torch.from_numpy(v[0]).cuda()
    dys = [torch.from_numpy(v[j + 1]).cuda() for j in range(nv)]
    sabs = np.array([np.sum(np.abs(v[0] * v[j + 1])) for j in range(nv)])
    ref = torch.zeros(nv, dtype=torch.float64, device="cuda")
    bdfb.nv_dot_prod_multi(dx, dys, ref, bdfb.nv_work(n, nv))
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        assert noalloc(dx, dys, outs[call], stream) == bdfb.SUCCESS
        torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # no device memory was taken
    for call in range(2):
        diff = np.abs(outs[call].cpu().numpy() - ref.cpu().numpy())
        assert np.all(diff <= 1e-14 * sabs), (call, diff)


def test_noalloc_rejects_too_many_vectors():
    nmax = int(L.bdfb_nv_noalloc_max_nv())
    assert nmax == 16
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(nmax + 1, dtype=torch.float64, device="cuda")
    assert noalloc(x, [x] * (nmax + 1), out, None) == bdfb.ILL_INPUT
