"""Automatic parameters (Sec. 4.3): the output-size estimate by random pair
sampling, the rule applied to it, and a whole run in automatic mode."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

COS = 0


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


def test_output_estimate_matches_exhaustive_count(msm):
    wl = W.WORKLOADS["small"]
    X = _t(W.clustered(wl.n, wl.dim, wl.n_clusters, wl.sigma, wl.data_seed))
    exact = msm.eps_count_exhaustive(X, COS, wl.eps)
    m = 1 << 22
    S = msm.estimate_output(X, COS, wl.eps, samples=m, seed=3)
    # binomial sampling error of the hit fraction f = exact / C(n, 2):
    # relative sd = sqrt((1 - f) / (m f)); allow 5 sd
    f = exact / (wl.n * (wl.n - 1) / 2)
    assert abs(S / exact - 1) < 5 * np.sqrt((1 - f) / (m * f))
    assert msm.estimate_output(X, COS, wl.eps, samples=m, seed=3) == S   # seeded
    assert msm.estimate_output(X, COS, wl.eps, samples=m, seed=4) != S


def test_automatic_mode_uses_the_rule_and_misses_little(msm):
    wl = W.WORKLOADS["small"]
    Xh = W.clustered(wl.n, wl.dim, wl.n_clusters, wl.sigma, wl.data_seed)
    X = _t(Xh)
    truth = msm.eps_count_exhaustive(X, COS, wl.eps)
    pairs, dist, st = msm.eps_graph(X, COS, wl.eps, 0, 0, 0, Q=0, miss_ratio=1e-6, seed=9,
                                    out_mode=0)
    p = oracle.p_cosine(float(np.float32(wl.eps)))
    assert (st["ell"], st["k"], st["d"], st["Q"]) == oracle.choose_params(wl.n, p, 1e-6,
                                                                          st["S_est"])
    assert abs(st["S_est"] / truth - 1) < 0.05
    # no false pair; the measured missing ratio is far below the worst-case bound
    got = pairs.cpu().numpy().view(np.uint64)
    dv = oracle.dist(Xh, got[:: max(1, len(got) // 5000)], oracle.COSINE)
    assert np.all(dv <= np.float32(wl.eps))
    assert st["count"] <= truth and (truth - st["count"]) / truth <= 1e-5
