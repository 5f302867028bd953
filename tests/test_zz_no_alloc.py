"""The allocation-free top-k entry point (tfs_select_top_noalloc) against the ordinary
one. It exists for callers that cannot call cudaMalloc: a pipeline that must not
synchronise the device between launches, or a framework whose device memory belongs to
its own pool. Collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_N = 1 << 16
TFS_ERR_ARG = -1


def _noalloc():
    from paper_2510_19047_b300 import binding
    f = binding.load_library().tfs_select_top_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def test_no_alloc_top_k_matches_allocating_entry_point():
    import torch
    from paper_2510_19047_b300.binding import TFS
    f = _noalloc()
    ctx = TFS(0)
    rng = np.random.default_rng(11)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row share the static scratch; the second must not see the first
    for n, k in ((MAX_N, 655), (40_000, 4000)):
        x = np.round(rng.normal(size=n), 3)  # many ties: order by lower index
        xd = torch.from_numpy(x).cuda()
        out = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        rc = f(ctypes.c_void_p(xd.data_ptr()), n, k, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ctx.select_top(x, k))
        # and against an order computed independently: value descending, index ascending
        assert np.array_equal(out.cpu().numpy(), np.lexsort((np.arange(n), -x))[:k])


def test_no_alloc_top_k_edge_cases_and_no_allocation():
    """k = n, NaN (ranked below every number), -0.0 tied with +0.0 (by index); free
    device memory is the same before and after a call."""
    import torch
    f = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(12)
    n = 5000
    x = np.round(rng.normal(size=n), 1)
    x[::7] = -0.0
    x[3::11] = 0.0
    x[5::13] = np.nan
    xd = torch.from_numpy(x).cuda()
    want = np.lexsort((np.arange(n), -np.where(np.isnan(x), -np.inf, x),
                       np.isnan(x)))  # NaN last, then by value, then by index
    # one call first: a fresh process loads the kernels' code on its first launch
    warm = torch.empty(n, dtype=torch.int64, device="cuda")
    assert f(ctypes.c_void_p(xd.data_ptr()), n, n, ctypes.c_void_p(warm.data_ptr()), stream) == 0
    for k in (n, 17):
        out = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = f(ctypes.c_void_p(xd.data_ptr()), n, k, ctypes.c_void_p(out.data_ptr()), stream)
        torch.cuda.synchronize()
        assert rc == 0 and torch.cuda.mem_get_info()[0] == free0
        assert np.array_equal(out.cpu().numpy(), want[:k]), k


def test_no_alloc_top_k_rejects_what_it_cannot_hold():
    import torch
    f = _noalloc()
    big = torch.zeros(MAX_N + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert f(ctypes.c_void_p(big.data_ptr()), MAX_N + 1, 4, ctypes.c_void_p(out.data_ptr()),
             None) == TFS_ERR_ARG
    host = np.zeros(16)
    assert f(ctypes.c_void_p(host.ctypes.data), 16, 4, ctypes.c_void_p(out.data_ptr()),
             None) == TFS_ERR_ARG
