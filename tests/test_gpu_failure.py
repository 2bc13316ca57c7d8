"""Failure paths, tested without faulting the GPU.

Allocation failure: a caller allocator that returns NULL on its k-th call
must make msm_eps_graph return MSM_E_NOMEM with every buffer it had
obtained released (no leak), and the next call must give the right result.

Bounded waits: with the poll limit of the tensor-core projection's waits set
to one poll (a testing knob, msm_set_wait_limit), the waits run out before
the first copy lands; the kernel then stops, waits for what it issued,
releases its tensor memory and reports it, so msm_project returns
MSM_E_TIMEOUT.  With the limit restored the next projection is bit-exact.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

MSM_E_NOMEM, MSM_E_TIMEOUT = -2, -5


@pytest.fixture(scope="module")
def msm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0904_3151_gb300 import build as b
    b.build()
    import paper_0904_3151_gb300 as m
    m.lib()
    return m


class FailingAllocator:
    """Device memory from PyTorch; the fail_at-th allocation returns NULL."""

    def __init__(self, fail_at):
        import torch
        from paper_0904_3151_gb300 import _lib
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self._a = _lib.ALLOC_FN(self._alloc)
        self._f = _lib.FREE_FN(self._free)
        self.struct = _lib.Allocator(self._a, self._f, None)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, stream, ctx):
        self.live.pop(ptr, None)


def _eps_graph_raw(msm, Xg, R, alloc, wl_args):
    import torch
    from paper_0904_3151_gb300 import _lib
    ell, k, d, Q, eps = wl_args
    p = _lib.Params()
    p.ell, p.k, p.d, p.Q = ell, k, d, Q
    p.R = R.data_ptr()
    p.out_mode = 0
    p.flags = 1  # canonical order
    out = _lib.Pairs()
    n, dim = Xg.shape
    st = msm.lib().msm_eps_graph(ctypes.c_void_p(Xg.data_ptr()), n, dim, 0, 0,
                                 ctypes.c_float(eps), ctypes.c_double(1e-6), ctypes.byref(p),
                                 ctypes.byref(alloc.struct), ctypes.byref(out), None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_allocation_failure_releases_everything(msm):
    import torch
    n, dim, args = 3000, 64, (64, 8, 4, 3, 0.15)
    X = W.clustered(n, dim, 15, 0.05, 41)
    R = W.gaussian_R(3, dim, 64, 42)
    Xg, Rg = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
    want, _, _ = oracle.eps_graph(X, R, 64, 8, 4, oracle.COSINE, 0.15)
    good = FailingAllocator(0)
    st, out = _eps_graph_raw(msm, Xg, Rg, good, args)
    assert st == 0
    total = good.calls
    assert total >= 5
    got = torch.empty(out.count, dtype=torch.int64, device="cuda")
    got.copy_(good.live[out.pairs].view(torch.int64)[:out.count])
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)
    for k in sorted({1, 2, total // 2, total - 1, total}):
        bad = FailingAllocator(k)
        st, out = _eps_graph_raw(msm, Xg, Rg, bad, args)
        torch.cuda.synchronize()
        assert st == MSM_E_NOMEM, (k, st, msm.lib().msm_last_error())
        assert bad.live == {}, f"allocation {k} failed: {len(bad.live)} buffers not released"
        assert out.count == 0
    # and a clean call afterwards
    again = FailingAllocator(0)
    st, out = _eps_graph_raw(msm, Xg, Rg, again, args)
    assert st == 0 and out.count == len(want)


def test_projection_wait_timeout_then_recovery(msm):
    import torch
    L = msm.lib()
    n, dim, ell, Q = 2000, 128, 128, 2
    X = W.clustered(n, dim, 7, 0.2, 5, normalise=False)
    R = W.gaussian_R(Q, dim, ell, 6)
    Xg, Rg = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
    old = L.msm_set_wait_limit(1)
    try:
        with pytest.raises(msm.MSMError) as e:
            msm.project(Xg, ell, Q, R=Rg)
        assert e.value.status == MSM_E_TIMEOUT
        torch.cuda.synchronize()
    finally:
        L.msm_set_wait_limit(0)
    assert old == 1 << 22
    S = msm.project(Xg, ell, Q, R=Rg)
    assert np.array_equal(S.cpu().numpy().view(np.uint64).reshape(Q, n, -1), oracle.project(X, R))
