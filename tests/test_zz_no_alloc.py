"""msm_recheck_noalloc: the epsilon recheck for callers that must not
allocate device memory (for example code inside a host application whose
allocator already owns the GPU).  It keeps its scratch in a static device
array, so these tests check, through the C ABI, that two calls in a row give
the same result as the ordinary msm_recheck entry point -- the second with a
different input and metric, so nothing left in the shared array from the
first call can leak into it -- that the kept pairs and distances equal the
CPU oracle's, that a failed call (zero row, out-of-range pair) leaves no
stale flag behind for the next call, and that oversize inputs are refused.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0904_3151_gb300 import build as b
    b.build()
    import paper_0904_3151_gb300 as m
    m.lib()
    return m


def _case(n, dim, metric, eps, seed):
    X = W.clustered(n, dim, 12, 0.05, seed)
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, 60000)
    j = rng.integers(0, n, 60000)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    keep = lo < hi
    cand = np.unique((lo[keep].astype(np.uint64) << np.uint64(32)) | hi[keep].astype(np.uint64))
    return X, cand


def _noalloc_status(msm, Xg, cand_g, metric, eps):
    """Call the no-alloc entry point directly through the C ABI with
    caller-owned outputs; returns (status, pairs, dist)."""
    import torch
    n, dim = Xg.shape
    m = cand_g.numel()
    pairs = torch.empty(max(m, 1), dtype=torch.int64, device=Xg.device)
    dist = torch.empty(max(m, 1), dtype=torch.float32, device=Xg.device)
    cnt = ctypes.c_int64(-1)
    rec = ctypes.c_int64(-1)
    st = msm.lib().msm_recheck_noalloc(
        ctypes.c_void_p(Xg.data_ptr()), n, dim, 0, metric, ctypes.c_float(eps),
        ctypes.c_void_p(cand_g.data_ptr()), m, ctypes.c_void_p(pairs.data_ptr()),
        ctypes.c_void_p(dist.data_ptr()), ctypes.byref(cnt), ctypes.byref(rec),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    k = max(cnt.value, 0)
    return st, pairs[:k], dist[:k]


def _noalloc(msm, Xg, cand_g, metric, eps):
    st, p, d = _noalloc_status(msm, Xg, cand_g, metric, eps)
    assert st == 0, msm.lib().msm_last_error()
    return p, d


def _sorted(p, d):
    p = p.cpu().numpy().view(np.uint64)
    d = d.cpu().numpy().astype(np.float64)
    o = np.argsort(p)
    return p[o], d[o]


def test_noalloc_matches_recheck_twice(msm):
    import torch
    for n, dim, metric, eps, seed in [(6000, 96, 0, 0.02, 31), (9000, 64, 1, 0.25, 32)]:
        X, cand = _case(n, dim, metric, eps, seed)
        Xg = torch.from_numpy(X).cuda()
        cg = torch.from_numpy(cand.view(np.int64)).cuda()
        ref_p, ref_d, _ = msm.recheck(Xg, cg, metric, eps)
        rp, rd = _sorted(ref_p, ref_d)
        assert len(rp) > 100
        gp, gd = _sorted(*_noalloc(msm, Xg, cg, metric, eps))
        assert np.array_equal(gp, rp)
        assert np.allclose(gd, rd, rtol=1e-5, atol=(dim + 8) * 2.0 ** -51)
        # and directly against the oracle's double-precision distances
        od = oracle.dist(X, cand, metric)
        ok = od <= np.float64(np.float32(eps))
        assert np.array_equal(gp, cand[ok])
        assert np.allclose(gd, od[ok], rtol=1e-5, atol=(dim + 8) * 2.0 ** -51)


def test_noalloc_failed_calls_leave_no_stale_flags(msm):
    """A call that fails (an all-zero row under cosine, then a candidate
    outside i < j < n) must not poison the shared array: the next clean call
    returns status 0 and the pairs of msm_recheck."""
    import torch
    X, cand = _case(5000, 64, 0, 0.02, 33)
    Xz = X.copy()
    Xz[17] = 0.0
    cg = torch.from_numpy(cand.view(np.int64)).cuda()
    st, _, _ = _noalloc_status(msm, torch.from_numpy(Xz).cuda(), cg, 0, 0.02)
    assert st == -6, msm.lib().msm_last_error()
    Xg = torch.from_numpy(X).cuda()
    bad = np.append(cand, np.uint64((7 << 32) | 5000))  # j = n
    st, _, _ = _noalloc_status(msm, Xg, torch.from_numpy(bad.view(np.int64)).cuda(), 0, 0.02)
    assert st == -1 and b"i < j < n" in msm.lib().msm_last_error()
    ref_p, ref_d, _ = msm.recheck(Xg, cg, 0, 0.02)
    rp, rd = _sorted(ref_p, ref_d)
    gp, gd = _sorted(*_noalloc(msm, Xg, cg, 0, 0.02))
    assert len(rp) > 100 and np.array_equal(gp, rp)
    assert np.allclose(gd, rd, rtol=1e-5, atol=72 * 2.0 ** -51)


def test_noalloc_refuses_oversize_input(msm):
    import torch
    n = (1 << 18) + 1
    Xg = torch.ones((n, 1), dtype=torch.float32, device="cuda")
    cg = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    cnt = ctypes.c_int64(0)
    st = msm.lib().msm_recheck_noalloc(
        ctypes.c_void_p(Xg.data_ptr()), n, 1, 0, 1, ctypes.c_float(0.1),
        ctypes.c_void_p(cg.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), None,
        ctypes.byref(cnt), None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
    assert b"at most" in msm.lib().msm_last_error()
