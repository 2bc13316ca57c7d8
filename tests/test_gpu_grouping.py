"""The grouping sort (steps A3-A4) on the paths its bucket sizes select.

With one point set, a top-digit pass splits every grouping into 256 buckets
and each bucket is sorted by one CTA: in shared memory when it holds at most
8192 items, else in chunks through a scratch copy.  These tests build pools
whose buckets exceed that capacity and check the pair lists: against the
CPU oracle where it finishes in seconds, and on 3,000,000 strings against
the same pool run as one set of a two-set call (the LSD path of the batched
form, itself checked against the oracle elsewhere).
"""
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


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_one_group_larger_than_shared_memory(msm):
    """10,000 strings share blocks 0-2 (one group of the kept set {0, 1, 2},
    k = 4, d = 1: a bucket of more than 8,192 items) and differ at random in
    block 3; 10,000 more are random.  Pairs equal the oracle's."""
    rng = np.random.default_rng(7)
    n = 20000
    S = W.random_strings(n, 64, 1, 8)
    S[0, :10000, 0] = (S[0, :10000, 0] & np.uint64(0xFFFF000000000000)) | np.uint64(0x0000A5A5C3C35A5A)
    got, st = msm.enumerate_pairs(_t(S.view(np.int64)), 64, 4, 1, canonical=True)
    want, ost = oracle.msm(S, 64, 4, 1)
    assert np.array_equal(_u64(got), want)
    # the kept blocks (48 bits) are grouped by a hashed key, whose collisions
    # can only add inspected pairs
    assert st["checks"] >= ost["checks"] >= 10000 * 9999 // 2


def test_large_buckets_match_the_set_path(msm):
    """3,000,000 clustered 64-bit strings (k = 8, d = 4): every top-digit
    bucket holds ~11,700 items, so every one takes the chunked path.  The
    same pool as the first set of a two-set call (the second empty) takes the
    LSD path; both must report the same pairs and inspect the same pairs."""
    n = 3_000_000
    S = W.clustered_words(n, 1, 11, n_centres=300_000, and_depth=5)
    Sg = _t(S.view(np.int64))
    p1, st1 = msm.enumerate_pairs(Sg, 64, 8, 4, canonical=True)
    p2, st2 = msm.enumerate_sets(Sg, [0, n, n], 64, 8, 4, canonical=True)
    a, b = _u64(p1), _u64(p2)
    assert len(a) > 1_000_000
    assert np.array_equal(a, b)
    assert st1["checks"] == st2["checks"]
